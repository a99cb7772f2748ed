#!/usr/bin/env python3
"""Throughput of the FNO SA-DSRG-PT2 hot path on GB300.

One step = one whole solve of the workload: vv-class PT2 energy and D_vv
(Eq. A12), natural orbitals (Eq. 8), and for every FNO cut the truncation
(Eq. 10 with the near-degeneracy rule) and the discarded-virtual correction
(Eq. 11, scalar part).  Inputs are seeded synthetic problems shaped like the
paper's workloads; B is resident in HBM before the timed region and is larger
than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched through torch.distributed.run) every rank solves its own
copy of the workload (replicas: the path needs no exchange on one problem);
value = solves of all ranks / max wall time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time
import types

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "sa_cas10_ncore60_nvir1200_naux3600"
# 64 independent instances of ragged size (synth.problems.batch_sizes, seed 3)
BATCH_WORKLOAD = "ragged_batch64_seed3"
BATCH_CUT = 98.5
PHASES = ("sliced_gemm_pair", "sliced_gemm_syrk", "sliced_gemm_plain", "phase_stage_b", "phase_pair_epilogue",
          "phase_dress", "phase_stage_sig", "phase_small_terms", "phase_no_eigen", "phase_density_eigen",
          "phase_recanon_and_rotate")
COUNTERS = ("eig_sweeps_large", "eig_sweeps_small")
METRIC = "DSRG-PT2 D_vv+E2 solves/sec & GFLOP/s, fast vs FP64 GPU form at ≤1e-7 Eh"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--nslices", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the float64 GPU form (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the sub-results (CAS(12,12) workload and the 64-instance batch)")
    ap.add_argument("--clock-ms", type=int, default=200,
                    help="nvidia-smi sampling interval during the timed steps (ms)")
    ap.add_argument("--fused-epilogue", action="store_true",
                    help="run the Eq. A7 regulariser in the contraction kernel (comparison with the separate default)")
    return ap.parse_args()


def max_over_ranks(x, dist, device):
    """Largest value of `x` over the ranks (the slowest replica sets the time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, world, ms_max):
    """Whole-job throughput of weakly scaled replicas: all ranks' units over
    the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def algorithmic_flops(p):
    """F_V + F_D per solve: naux nvir^2 nh (nh+1) + nh^2 nvir^3."""
    nh = p.ncore + p.nact
    return float(p.naux) * p.nvir ** 2 * nh * (nh + 1) + float(nh) ** 2 * p.nvir ** 3


def pair_alg_flops(p, nkept):
    """Algorithmic flops of the pair contractions of one solve (the count of
    the measurement plan): 2 naux nv^2 per unordered hole pair (i <= j), for
    the D_vv pass (nv = nvir) and for the energy pass of every FNO cut
    (nv = N')."""
    nh = p.ncore + p.nact
    pairs = nh * (nh + 1) / 2
    return sum(2.0 * p.naux * float(v) ** 2 * pairs for v in [p.nvir] + list(nkept))


def cut_margins(ons, p_o, nkept, degen_ratio=0.01):
    """How far the p_o cut was from moving: with c(k) the cumulative ON
    fraction of the k largest ONs and k0 the smallest k with c(k) >= p_o/100,
    above = c(k0) - p_o/100 and below = p_o/100 - c(k0 - 1); the widening then
    adds ONs while the relative gap to the next one is below degen_ratio, and
    stop_gap is that relative gap where it stopped (N' = nkept)."""
    import numpy as np
    n = np.asarray(ons, dtype=np.float64)
    c = np.cumsum(n) / np.sum(n)
    t = p_o / 100.0
    k0 = int(np.nonzero(c >= t)[0][0]) + 1 if np.any(c >= t) else len(n)
    out = {"p_o": p_o, "nkept": int(nkept), "k0": k0, "above": float(c[k0 - 1] - t),
           "below": float(t - (c[k0 - 2] if k0 >= 2 else 0.0)), "widened_by": int(nkept - k0)}
    if 0 < nkept < len(n):
        a, b = n[nkept - 1], n[nkept]
        out["stop_gap"] = float((a - b) / max(a, b))
        out["degen_ratio"] = degen_ratio
    return out


def cuts_of(name):
    from synth import CUTS
    return CUTS.get(name, (98.5,))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, device_index: int, interval_ms: int = 200):
        self.dev = device_index
        self.interval = max(int(interval_ms), 50)
        self.lines = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", str(self.interval)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
class OracleSample:
    """Stratified timing of one oracle solve (oracle.solve: E_vv, D_vv terms
    1-12, NOs, and per cut the FNO problem and its E_vv) on the host cores.

    The solve's work falls into strata whose unit costs differ; each stratum
    is timed on a sample of its units through the oracle's own functions, and
    the solve's time is the sum of unit time x unit count:
      amp     semi-internal amplitudes for a subset of the holes (cost ~ holes^2) and T1
      small   Eq. A12 terms 1-3, 6, 8-12 (whole)
      cc      core pairs m < n: E_vv group {mn, nm} and term 4; m = n likewise
      ca      core m: E_vv group {mu, um}_u; term 5 = its amplitude blocks
              + one unit per active u (two calls separate the two)
      aa      active pairs: E_vv group; term 7 = its amplitude blocks + one
              unit per (u, v) (two calls)
      no      NOs of a symmetric nvir x nvir matrix
      corr    per cut: recanonicalisation, the rotated problem, and E_vv of
              a sample of its groups (by kind, scaled by counts)
    The semi-internal amplitudes and T1 of the whole problem, built once per
    process outside the timed samples, feed the term samples.  Groups of
    strata are timed one at a time (`run_group`), so a step can stay short."""

    def __init__(self, p, nkept):
        import oracle as O
        self.O, self.p = O, p
        self.nkept = [int(k) for k in nkept]
        nc, na = p.ncore, p.nact
        self.ts = O.t2_semi_internal(p) if na else None
        self.t1 = O.t1_amplitudes(p, self.ts)
        self.unit = {}      # stratum -> measured seconds per unit (latest)
        self.count = {}     # stratum -> units per solve
        groups = [["amp", "small", "no"], ["cc"]]
        if na:
            groups += [["ca_evv"], ["ca_t5a"], ["ca_t5b"], ["aa_evv"], ["aa_t7a"], ["aa_t7b"]]
        groups += [[f"corr{i}"] for i in range(len(self.nkept))]
        self.groups = groups
        self.next = 0

    def _t(self, f):
        t0 = time.perf_counter()
        f()
        return time.perf_counter() - t0

    def _stratum(self, name):
        O, p = self.O, self.p
        nc, na, nh = p.ncore, p.nact, p.ncore + p.nact
        ts, t1 = self.ts, self.t1
        if name == "amp":
            k = max(1, min(nh, int(round(nh / 5))))
            h = list(range(0, nh, max(1, nh // k)))[:k]
            dt = self._t(lambda: O.t2_semi_internal(p, holes=h)) if na else 0.0
            dt += self._t(lambda: O.t1_amplitudes(p, ts))
            self.unit["amp"], self.count["amp"] = dt, 1.0
            if na:   # the amplitude build scales with the ordered hole pairs
                self.unit["amp"] = dt * (nh / len(h)) ** 2
            return dt
        if name == "small":
            dt = self._t(lambda: O.dvv_terms(p, terms=(1, 2, 3, 6, 8, 9, 10, 11, 12), ts=ts, t1=t1))
            self.unit["small"], self.count["small"] = dt, 1.0
            return dt
        if name == "no":
            rng = __import__("numpy").random.default_rng(0)
            a = rng.standard_normal((p.nvir, p.nvir))
            d = a + a.T
            dt = self._t(lambda: O.natural_orbitals(d))
            self.unit["no"], self.count["no"] = dt, 1.0
            return dt
        if name == "cc":
            dt = 0.0
            off = [(m, (m + 1 + 7 * m) % nc) for m in range(0, nc, max(1, nc // 3))][:3] if nc > 1 else []
            off = [(min(a, b), max(a, b)) for a, b in off if a != b]
            for (m, n) in off:
                dt_p = self._t(lambda: O.e_vv(p, components=[[(m, n), (n, m)]]))
                dt_p += self._t(lambda: O.dvv_terms(p, terms=(4,), ts=ts, t1=t1, core_pairs=[(m, n)]))
                dt += dt_p
            if off:
                self.unit["cc_off"] = dt / len(off)
                self.count["cc_off"] = nc * (nc - 1) / 2
            m = nc // 2
            dd = self._t(lambda: O.e_vv(p, components=[[(m, m)]]))
            dd += self._t(lambda: O.dvv_terms(p, terms=(4,), ts=ts, t1=t1, core_pairs=[(m, m)]))
            self.unit["cc_diag"], self.count["cc_diag"] = dd, float(nc)
            return dt + dd
        m = nc // 2
        if name == "ca_evv":
            comp = [(m, nc + u) for u in range(na)] + [(nc + u, m) for u in range(na)]
            dt = self._t(lambda: O.e_vv(p, components=[comp]))
            self.unit["ca_evv"], self.count["ca_evv"] = dt, float(nc)
            return dt
        if name in ("ca_t5a", "ca_t5b"):
            sel = [(m, 0)] if name == "ca_t5a" else [(m, 1 % na), (m, 2 % na)]
            sel = list(dict.fromkeys(sel))
            dt = self._t(lambda: O.dvv_terms(p, terms=(5,), ts=ts, t1=t1, ca_pairs=sel))
            self.unit[name] = (dt, len(sel))
            self._split("ca_t5", nc, na)
            return dt
        if name == "aa_evv":
            comp = [(nc + u, nc + v) for u in range(na) for v in range(na)]
            dt = self._t(lambda: O.e_vv(p, components=[comp]))
            self.unit["aa_evv"], self.count["aa_evv"] = dt, 1.0
            return dt
        if name in ("aa_t7a", "aa_t7b"):
            sel = [(0, 0)] if name == "aa_t7a" else [(0, 1 % na), (1 % na, 0)]
            sel = list(dict.fromkeys(sel))
            dt = self._t(lambda: O.dvv_terms(p, terms=(7,), ts=ts, t1=t1, aa_pairs=sel))
            self.unit[name] = (dt, len(sel))
            self._split("aa_t7", 1, na * na)
            return dt
        if name.startswith("corr"):
            return self._corr(int(name[4:]))
        raise KeyError(name)

    def _split(self, key, groups, units):
        """Two timings with 1 and 2 units: fixed part per group + per-unit part."""
        a, b = self.unit.get(key + "a"), self.unit.get(key + "b")
        if not a or not b:
            return
        (ta, na_), (tb, nb) = a, b
        per = max(0.0, (tb - ta) / max(nb - na_, 1)) if nb != na_ else ta / na_
        fixed = max(0.0, ta - na_ * per)
        self.unit[key] = fixed + units * per
        self.count[key] = float(groups)

    def _corr(self, i):
        O, p = self.O, self.p
        import numpy as np
        k = self.nkept[i]
        rng = np.random.default_rng(1 + i)
        q, _ = np.linalg.qr(rng.standard_normal((p.nvir, p.nvir)))
        t0 = time.perf_counter()
        U, eps_new = O.recanonicalize(p, q, k)
        pf = O.fno_problem(p, U, eps_new)
        comps = O.hole_pair_components(pf)
        fixed = time.perf_counter() - t0
        kinds = {}
        for c in comps:
            kinds.setdefault(len(c), []).append(c)
        dt = fixed
        est = fixed
        for size, cs in kinds.items():
            take = cs[:: max(1, len(cs) // 3)][:3]
            t = self._t(lambda: O.e_vv(pf, components=take))
            dt += t
            est += t / len(take) * len(cs)
        self.unit[f"corr{i}"], self.count[f"corr{i}"] = est, 1.0
        return dt

    def run_group(self):
        """Times the next group of strata; returns the seconds measured."""
        g = self.groups[self.next % len(self.groups)]
        self.next += 1
        return sum(self._stratum(nm) for nm in g)

    def complete(self):
        return self.next >= len(self.groups)

    def solve_seconds(self):
        return sum(v * self.count[k] for k, v in self.unit.items() if k in self.count and not isinstance(v, tuple))


def _oracle_cores():
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max(i.get("num_threads", 1) for i in threadpool_info()) or cores
    except Exception:
        pass
    return cores


def cpu_baseline(p, nkept):
    """The oracle as it stands on the host cores: one stratified sample of a
    whole solve (OracleSample, every group once), extrapolated to solves/s."""
    s = OracleSample(p, nkept)
    measured = 0.0
    while not s.complete():
        measured += s.run_group()
    sec = s.solve_seconds()
    return {"value": 1.0 / sec, "unit": "solves/s", "cores": _oracle_cores(), "kind": "oracle",
            "sample": f"stratified sample of one oracle solve ({len(s.groups)} groups of strata: amplitudes, "
                      f"small terms, core pairs, core-active groups, active pairs, NOs, {len(nkept)} FNO "
                      f"corrections), {measured:.1f} s timed, extrapolated by unit counts to {sec:.0f} s "
                      f"per solve"}


def batch_cpu_baseline(nkept_by_instance):
    """The oracle's stratified sample on the largest instance of the ragged
    batch, rescaled from that instance's flops to the batch's mean
    (instances per second of the whole 64-instance mix)."""
    from synth.problems import batch_sizes, batch_problem
    sizes = batch_sizes()
    fl = [algorithmic_flops(types.SimpleNamespace(**s)) for s in sizes]
    k = max(range(len(sizes)), key=lambda i: fl[i])
    r = cpu_baseline(batch_problem(k), [nkept_by_instance[k]])
    flops_per_s = r["value"] * fl[k]
    r["value"] = flops_per_s / (sum(fl) / len(fl))
    r["unit"] = "instances/s"
    r["sample"] = f"instance {k} of the batch (largest): " + r["sample"] + "; rescaled by the batch's mean flops"
    return r


def reference_nkept(name, p):
    """N' per cut for the correction strata of the reference arm: the stored
    oracle values of the workload when present, else 15 % of nvir."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    cuts = cuts_of(name)
    try:
        with open(path) as f:
            g = json.load(f)
        return [int(g["cuts"][str(c)]["nkept"]) for c in cuts]
    except (OSError, KeyError, ValueError):
        return [max(1, int(0.15 * p.nvir)) for _ in cuts]


def single_config(p, name, cuts, nslices):
    """`config` of a single-workload line (both arms)."""
    return {"workload": name, "ncore": p.ncore, "nact": p.nact, "nvir": p.nvir, "naux": p.naux,
            "nstates": len(p.weights), "s": p.s, "cuts_po": list(cuts), "nslices": nslices,
            "l2": f"inputs larger than L2 (B = {p.B.nbytes / 1e9:.2f} GB)", "parallelism": "replicas"}


def batch_config(nslices):
    """`config` of a batch line (both arms): the shape recipe of the 64 instances."""
    from synth.problems import batch_sizes
    sizes = batch_sizes()
    bbytes = sum(8 * s["naux"] * (s["ncore"] + s["nact"]) * (s["nact"] + s["nvir"]) for s in sizes)
    return {"workload": BATCH_WORKLOAD, "instances": len(sizes), "ncore": "U{10..60}", "nact": "{0,4,6,8}",
            "nvir": "U{100..800}", "naux": "3 (ncore+nact+nvir)", "nstates": "2..5",
            "cut_po": BATCH_CUT, "nslices": nslices,
            "l2": f"inputs larger than L2 ({bbytes / 1e9:.1f} GB of B)", "parallelism": "replicas"}


def reference_arm(args):
    """The oracle timed on the host cores.  A step times one group of strata
    of OracleSample (a bounded sample of the workload's solve); groups rotate
    over the warm-up and timed steps, and the value is the solves/s of the
    whole solve extrapolated from the latest timing of every stratum.
    ms_per_step is the measured length of a timed step."""
    from synth import workload
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    batch = args.workload == BATCH_WORKLOAD
    if batch:
        from synth.problems import batch_sizes, batch_problem
        sizes = batch_sizes()
        fl = [algorithmic_flops(types.SimpleNamespace(**sz)) for sz in sizes]
        k = max(range(len(sizes)), key=lambda i: fl[i])
        p = batch_problem(k)
        nk = [max(1, int(0.15 * p.nvir))]
        config = batch_config(args.nslices)
        scale = fl[k] / (sum(fl) / len(fl))
        unit = "instances/s"
    else:
        p = workload(args.workload)
        nk = reference_nkept(args.workload, p)
        config = single_config(p, args.workload, cuts_of(args.workload), args.nslices)
        scale = 1.0
        unit = "solves/s"
    s = OracleSample(p, nk)
    for _ in range(args.warmup):
        s.run_group()
    times = [s.run_group() for _ in range(args.steps)]
    while not s.complete():
        s.run_group()
    v = scale / s.solve_seconds()
    sample = (f"one group of strata of a stratified oracle solve per step ({len(s.groups)} groups rotate), "
              f"extrapolated by unit counts to {s.solve_seconds():.0f} s per solve"
              + ("; largest batch instance, rescaled by the batch's mean flops" if batch else ""))
    ms = 1e3 * sum(times) / max(len(times), 1)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": v, "unit": unit, "cores": _oracle_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == BATCH_WORKLOAD:
        batch_arm(args)
        return
    import numpy as np
    import torch

    import paper_2312_07008_gb300 as pkg
    from synth import workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    p = workload(args.workload)
    cuts = cuts_of(args.workload)
    nv = p.nvir
    pkg.dsrg_fno_debug_set_fused_epilogue(args.fused_epilogue)
    dev = torch.device("cuda", local)
    gp = pkg.problem_from_synth(p, dev, pkg.SLICED_BF16, args.nslices)
    d = torch.empty((nv, nv), dtype=torch.float64, device=dev)
    on = torch.empty(nv, dtype=torch.float64, device=dev)
    no = torch.empty((nv, nv), dtype=torch.float64, device=dev)

    def step(prob, after_d=None):
        e2 = pkg.dsrg_fno_vv_opdm(prob, d)
        if after_d is not None:  # end to end: the next step's input copy starts here
            after_d()
        res = {"e2": e2}
        for i, c in enumerate(cuts):
            if i == 0:   # NOs once, then every cut of the same ONs
                k = pkg.dsrg_fno_truncate(nv, d, pkg.MODE_PO, c, 0.01, on, no)
            else:
                k = pkg.dsrg_fno_cut(nv, on, pkg.MODE_PO, c, 0.01)
            de, ef = pkg.dsrg_fno_discarded_correction(prob, k, no, e2_mo=e2)
            res[c] = (k, de)
        return res

    for _ in range(args.warmup):
        step(gp)
    stream = torch.cuda.current_stream()
    barrier()
    clk = ClockSampler(local, args.clock_ms)
    clk.start()
    time.sleep(0.3)
    pkg.dsrg_fno_launch_count(reset=True)
    pkg.dsrg_fno_profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        res = step(gp)
    ev1.record(stream)
    barrier()
    pkg.dsrg_fno_profile_enable(False)
    launches = pkg.dsrg_fno_launch_count()
    ms = ev0.elapsed_time(ev1)
    phases = {}
    for nm in PHASES:
        t_ms, n_l, _ = pkg.dsrg_fno_profile_query(nm)
        phases[nm] = {"ms_per_step": t_ms / args.steps, "launches_or_calls": n_l}
    for nm in COUNTERS:
        _, n_c, total = pkg.dsrg_fno_profile_query(nm)
        phases[nm] = {"calls": n_c, "mean": total / max(n_c, 1)}
    ons_last = on.cpu().numpy()
    pair_ms, pair_n, pair_fl = pkg.dsrg_fno_profile_query("sliced_gemm_pair")
    syrk_ms, syrk_n, syrk_fl = pkg.dsrg_fno_profile_query("sliced_gemm_syrk")
    plain_ms, plain_n, plain_fl = pkg.dsrg_fno_profile_query("sliced_gemm_plain")
    ms_max = max_over_ranks(ms, dist, dev)
    value = replica_rate(args.steps, world, ms_max)
    flops = algorithmic_flops(p)

    # ---- end to end through the C ABI, host buffers in pinned memory: every
    # step copies its inputs from pinned host memory into one of two device
    # input sets on a copy stream and reads its ONs back into pinned host
    # memory.  The copy of step i + 1 is issued once step i's D pass has
    # returned, so that it runs beside the latency-bound eigensolve and
    # corrections rather than the contraction kernels (C2: 735-787 ms per
    # step against 778-838 ms with the copy issued at the start of step i)
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
            for k, v in (("B", p.B), ("eps", p.eps), ("g1", p.gamma1), ("l2", p.lambda2)) if v is not None}
    sets = [{k: torch.empty_like(v, device=dev) for k, v in host.items()} for _ in range(2)]
    probs = [pkg.Problem(p.ncore, p.nact, p.nvir, p.naux, b["B"], b["eps"], b.get("g1"), b.get("l2"),
                         None, p.weights, p.s, pkg.SLICED_BF16, args.nslices) for b in sets]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    on_host = torch.empty(nv, dtype=torch.float64).pin_memory()
    d2h = on_host.numel() * 8 + 8 * (1 + 2 * len(cuts))
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def issue_copy(j):
        copy_stream.wait_event(freed[j])  # the step that last read input set j has finished
        with torch.cuda.stream(copy_stream):
            for k in host:
                sets[j][k].copy_(host[k], non_blocking=True)
        copied[j].record(copy_stream)

    def e2e_run(nsteps):
        for j in range(2):
            freed[j].record(stream)
        issue_copy(0)
        r = None
        for i in range(nsteps):
            j = i % 2
            nxt = (lambda: issue_copy(1 - j)) if i + 1 < nsteps else None
            stream.wait_event(copied[j])
            r = step(probs[j], nxt)
            freed[j].record(stream)
            on_host.copy_(on, non_blocking=True)
        torch.cuda.synchronize()
        return r

    e2e_run(2)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    barrier()
    e2e_value = replica_rate(args.steps, world, max_over_ranks(e0.elapsed_time(e1), dist, dev))
    clocks = clk.stop()  # sampled over the device-timed and the end-to-end steps

    # ---- the plain float64 GPU form of the same solve
    fp64 = None
    if args.fp64_steps > 0:
        gp64 = pkg.problem_from_synth(p, dev, pkg.FP64)
        step(gp64)
        barrier()
        pkg.dsrg_fno_profile_enable(True)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            r64 = step(gp64)
        f1.record(stream)
        barrier()
        pkg.dsrg_fno_profile_enable(False)
        fms = f0.elapsed_time(f1) / args.fp64_steps
        f64_ms, f64_n, _ = pkg.dsrg_fno_profile_query("pair_gemm_f64")
        f64_alg = pair_alg_flops(p, [r64[c][0] for c in cuts]) * args.fp64_steps
        f64_tf = f64_alg / (f64_ms / 1e3) / 1e12 if f64_ms > 0 else None
        fp64 = {"solves_per_s": 1e3 / fms, "s_per_solve": fms / 1e3, "gflops": flops / (fms / 1e3) / 1e9,
                "note": "contractions and elementwise stages in float64; the eigensolves run in double-float "
                        "(about 48 bits) in both forms",
                "roofline": {"bound": "fp64", "kernel": "pair_gemm_f64_kernel (float64 CUDA cores)",
                             "achieved": f64_tf, "unit": "TFLOP/s", "launches": f64_n,
                             "ms_per_step": f64_ms / args.fp64_steps,
                             "peak": PEAKS_OWN["fp64_dgemm_tflops"],
                             "peak_kind": "cuBLAS float64 GEMM (torch.matmul), measured by this repository",
                             "frac": (f64_tf / PEAKS_OWN["fp64_dgemm_tflops"])
                             if (f64_tf and PEAKS_OWN["fp64_dgemm_tflops"]) else None,
                             "frac_of_nominal": (f64_tf / 1.25) if f64_tf else None,
                             "nominal_tflops": 1.25},
                "fast_minus_fp64": {"e2": res["e2"] - r64["e2"],
                                    **{f"de_{c}": res[c][1] - r64[c][1] for c in cuts},
                                    **{f"nkept_{c}": [res[c][0], r64[c][0]] for c in cuts}}}

    alg = pair_alg_flops(p, [res[c][0] for c in cuts]) * args.steps
    roofline = roofline_of(pair_ms, pair_n, pair_fl, (syrk_ms, syrk_n, syrk_fl), (plain_ms, plain_n, plain_fl), ms,
                           args.workload, alg_flops=alg, nslices=args.nslices)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"bf16 digit planes (k={args.nslices}) -> exact f32 level sums -> f64",
        "data": "synthetic",
        "config": dict(single_config(p, args.workload, cuts, args.nslices),
                       epilogue="fused" if args.fused_epilogue else "separate kernel"),
        "gflops": flops * value / 1e9,
        "s_per_solve": ms_max / args.steps / 1e3,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "phases": phases,
        "clocks": clocks,
        "fp64_form": fp64,
        "result": {"e2": res["e2"], **{f"nkept_{c}": res[c][0] for c in cuts}, **{f"de_{c}": res[c][1] for c in cuts},
                   "cut_margins": [cut_margins(ons_last, c, res[c][0]) for c in cuts]},
    }
    if not args.no_sub:
        line["mr_energy"] = mr_energy_timing(pkg, p, gp, dev)
        line["sub_results"] = sub_results(pkg, dev, args.nslices)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, [res[c][0] for c in cuts])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def mr_energy_timing(pkg, p, gp, dev, steps=2):
    """The full second-order energy over every amplitude class
    (dsrg_fno_pt2_energy_mr) on the headline workload, with a seeded synthetic
    3-cumulant: E_vv on the digit-plane path, the rest (doubles with an active
    particle, singles, cumulant couplings) in float64; timed beside E_vv alone.
    rest_gemm_flops: the float64 integral GEMM of the rest, 2 nh np nh nact naux."""
    import torch
    from synth.problems import random_cumulant3
    l3 = torch.from_numpy(random_cumulant3(p.nact, 2)).to(dev) if p.nact else None
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps / 1e3, r

    s_full, (e2, evv) = timed(lambda: pkg.dsrg_fno_pt2_energy_mr(gp, l3))
    s_vv, _ = timed(lambda: pkg.dsrg_fno_pt2_energy(gp))
    # phases of one more call: the integral GEMM (digit planes) and the element stages of the rest
    pkg.dsrg_fno_profile_enable(True)
    pkg.dsrg_fno_pt2_energy_mr(gp, l3)
    torch.cuda.synchronize()
    pkg.dsrg_fno_profile_enable(False)
    ph = {nm: pkg.dsrg_fno_profile_query(nm)[0] / 1e3 for nm in ("phase_mr_integrals", "phase_mr_terms")}
    g_ms, _, g_fl = pkg.dsrg_fno_profile_query("sliced_gemm_plain")
    flops = 2.0 * p.nh * p.np_ * p.nh * p.nact * p.naux
    return {"s_full": s_full, "s_vv_only": s_vv, "s_rest": s_full - s_vv, "e2": e2, "e_vv": evv,
            "e_rest": e2 - evv, "lambda3": "seeded synthetic 3-cumulant (scale 0.03)", "steps": steps,
            "s_rest_integrals": ph["phase_mr_integrals"], "s_rest_terms": ph["phase_mr_terms"],
            "rest_gemm_flops": flops, "rest_gemm_ms": g_ms,
            "rest_gemm_tflops_executed": (g_fl / (g_ms / 1e3) / 1e12) if g_ms > 0 else None}


SUB_SINGLE = "sa_cas12_ncore95_nvir1000_naux4200"


def sub_results(pkg, dev, nslices, steps=3, warmup=2):
    """The other two measured workloads, timed after the headline one:
    the CAS(12,12) ncore 95 / nvir 1000 / naux 4200 solve (fast form) and
    the 64-instance ragged batch through dsrg_fno_batch_run."""
    import torch
    from synth import workload
    from synth.problems import batch_sizes, batch_problem
    out = {}
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n, r

    p = workload(SUB_SINGLE)
    cuts = cuts_of(SUB_SINGLE)
    nv = p.nvir
    gp = pkg.problem_from_synth(p, dev, pkg.SLICED_BF16, nslices)
    d = torch.empty((nv, nv), dtype=torch.float64, device=dev)
    on = torch.empty(nv, dtype=torch.float64, device=dev)
    no = torch.empty((nv, nv), dtype=torch.float64, device=dev)

    def one():
        e2 = pkg.dsrg_fno_vv_opdm(gp, d)
        res = {"e2": e2}
        for i, c in enumerate(cuts):
            k = (pkg.dsrg_fno_truncate(nv, d, pkg.MODE_PO, c, 0.01, on, no) if i == 0
                 else pkg.dsrg_fno_cut(nv, on, pkg.MODE_PO, c, 0.01))
            res[c] = (k, pkg.dsrg_fno_discarded_correction(gp, k, no, e2_mo=e2)[0])
        return res

    for _ in range(warmup):
        one()
    ms, r = timed(one, steps)
    out[SUB_SINGLE] = {"s_per_solve": ms / 1e3, "solves_per_s": 1e3 / ms,
                       "gflops": algorithmic_flops(p) / (ms / 1e3) / 1e9, "steps": steps, "warmup": warmup,
                       "e2": r["e2"], **{f"nkept_{c}": r[c][0] for c in cuts}, **{f"de_{c}": r[c][1] for c in cuts},
                       "cut_margins": [cut_margins(on.cpu().numpy(), c, r[c][0]) for c in cuts]}
    del gp, d, on, no
    sizes = batch_sizes()
    probs = [batch_problem(k) for k in range(len(sizes))]
    gps = [pkg.problem_from_synth(q, dev, pkg.SLICED_BF16, nslices) for q in probs]
    dvv = [torch.empty((q.nvir, q.nvir), dtype=torch.float64, device=dev) for q in probs]
    ons = [torch.empty(q.nvir, dtype=torch.float64, device=dev) for q in probs]
    nos = [torch.empty((q.nvir, q.nvir), dtype=torch.float64, device=dev) for q in probs]
    cut = (pkg.MODE_PO, BATCH_CUT, 0.01)
    run = lambda: pkg.dsrg_fno_batch_run(gps, dvv, cut, ons, nos, correction=True, nworkers=0)  # noqa: E731
    for _ in range(max(warmup, 4)):   # the first calls try 2, 4 and 8 workers
        run()
    ms, r = timed(run, steps)
    out[BATCH_WORKLOAD] = {"s_per_batch": ms / 1e3, "instances_per_s": len(probs) / (ms / 1e3),
                           "gflops": sum(algorithmic_flops(q) for q in probs) / (ms / 1e3) / 1e9,
                           "workers": pkg.dsrg_fno_batch_last_workers(), "steps": steps,
                           "sum_e2": sum(x["e2"] for x in r), "sum_nkept": sum(x["nkept"] for x in r)}
    del gps, dvv, ons, nos
    out["ladder_fno"] = ladder_timings(pkg, dev)
    out["naf"] = naf_timing(pkg, dev, nslices)
    return out


def ladder_timings(pkg, dev, nvs=(171, 203, 300), naux=3600, nh=70):
    """The particle-particle ladder of Eq. 6 for the hole pairs of the nvir
    1200 / naux 3600 workload (nh = 70: 2485 pairs i <= j) in virtual bases
    of the sizes the p_o = 98 % and 99 % cuts keep (171, 203) and one larger;
    seeded normal B_vv (symmetric in a, b) and amplitudes drawn on the device.
    The cost grows as nv^4: the fitted exponent and the extrapolated time of
    the untruncated basis (nvir 1200) are reported."""
    import math
    import torch
    npairs = nh * (nh + 1) // 2
    g = torch.Generator(device=dev)
    rows = []
    for nv in nvs:
        g.manual_seed(nv)
        Bv = 0.05 * torch.randn((naux, nv, nv), dtype=torch.float64, device=dev, generator=g)
        Bv = (Bv + Bv.transpose(1, 2)) / math.sqrt(2.0)
        T = 0.01 * torch.randn((npairs, nv, nv), dtype=torch.float64, device=dev, generator=g)
        C = torch.empty_like(T)
        pkg.dsrg_fno_ladder(Bv, T, C)   # warm-up (workspace)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pkg.dsrg_fno_ladder(Bv, T, C)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        flops = 2.0 * nv ** 4 * (naux + npairs)
        rows.append({"nv": nv, "ms": ms, "tflops_algorithmic": flops / (ms / 1e3) / 1e12})
        del Bv, T, C
    x = [math.log(r["nv"]) for r in rows]
    y = [math.log(r["ms"]) for r in rows]
    n = len(x)
    slope = (n * sum(a * b for a, b in zip(x, y)) - sum(x) * sum(y)) / (n * sum(a * a for a in x) - sum(x) ** 2)
    full = rows[-1]["ms"] * (1200.0 / rows[-1]["nv"]) ** 4
    return {"npairs": npairs, "naux": naux, "timings": rows, "fitted_exponent": slope,
            "extrapolated_ms_nvir1200": full,
            "speedup_at_nv203": full / next(r["ms"] for r in rows if r["nv"] == 203)}


def naf_timing(pkg, dev, nslices, keep_frac=0.75):
    """Natural auxiliary functions of the nvir 1200 / naux 3600 workload:
    time of dsrg_fno_naf keeping the largest 75 % of W's spectrum, and the
    PT2 energy of the compressed problem against the full one."""
    import torch
    from synth import workload
    p = workload(DEFAULT_WORKLOAD)
    nh, np_ = p.ncore + p.nact, p.nact + p.nvir
    B = torch.from_numpy(p.B).to(dev)
    Bo = torch.empty_like(B)
    w = torch.empty(p.naux, dtype=torch.float64, device=dev)
    pkg.dsrg_fno_naf(nh, np_, p.naux, B, 1e300, pkg.SLICED_BF16, Bo, w)   # spectrum only (nothing kept)
    ws = w.cpu().numpy()
    k_target = int(keep_frac * p.naux)
    thr = 0.5 * (ws[k_target - 1] + ws[k_target])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    k = pkg.dsrg_fno_naf(nh, np_, p.naux, B, thr, pkg.SLICED_BF16, Bo, w)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    gp = pkg.problem_from_synth(p, dev, pkg.SLICED_BF16, nslices)
    gq = pkg.Problem(p.ncore, p.nact, p.nvir, k, Bo[:k].contiguous(), gp.tensors[1], gp.tensors[2], gp.tensors[3],
                     None, p.weights, p.s, pkg.SLICED_BF16, nslices)
    e_full = pkg.dsrg_fno_pt2_energy(gp)
    torch.cuda.synchronize()
    c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c.record()
    e_naf = pkg.dsrg_fno_pt2_energy(gq)
    d.record()
    torch.cuda.synchronize()
    c2, d2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c2.record()
    pkg.dsrg_fno_pt2_energy(gp)
    d2.record()
    torch.cuda.synchronize()
    return {"naux": p.naux, "kept": k, "threshold": thr, "w_max": float(ws[0]), "w_min": float(ws[-1]),
            "naf_ms": ms, "e2_full": e_full, "e2_naf": e_naf, "energy_ms_naf": c.elapsed_time(d),
            "energy_ms_full": c2.elapsed_time(d2)}


# DRAM bytes per executed flop of the pair contraction, from one ncu capture
# of a small pair launch of the same kernel, scaled to this workload's
# launches; valid only for the kernel sources it was taken with.
TRAFFIC = {
    "sa_cas10_ncore60_nvir1200_naux3600": {
        # small-case capture (energy pass of ncore 20 / nact 4 / nvir 1100 / naux 2000):
        # 9.328 GB read + 2.908 GB written for 2.2556e13 executed flops
        "bytes_per_exec_flop": (9.328328e9 + 2.907642e9) / 2.2556379709440e13,
        "sha256": {"paper_2312_07008_gb300/csrc/sliced.cu":
                   "4ae42af7897f57e9271091737d32b7b3ac1c4d64dea612fe28a0ab301f83f347",
                   "paper_2312_07008_gb300/csrc/tc_ptx.cuh":
                   "300804d055c2a37a13d0d68e3e9d556e62027073a7a31151f5033bd4885f0757"},
    },
}


def traffic_per_launch(workload, exec_flops_per_launch):
    """DRAM bytes of an average pair launch, or None when no capture matches
    the current kernel sources."""
    import hashlib
    t = TRAFFIC.get(workload)
    if t is None:
        return None
    for rel, digest in t["sha256"].items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return t["bytes_per_exec_flop"] * exec_flops_per_launch


# Peaks this repository measured itself (MEASURED_PEAKS.json holds bf16 and
# HBM only): cuBLAS float64 and TF32 GEMMs through torch.matmul on one GB300,
# n = 8192, best of 5 or 10, CUDA events, SM clock at its 2070 MHz maximum.
PEAKS_OWN = {"fp64_dgemm_tflops": 1.0988, "tf32_tflops": 1027.07}


def roofline_of(pair_ms, pair_n, pair_fl, syrk, plain, step_ms, workload=None, alg_flops=None, nslices=5):
    """Roofline of the pair contraction (the dominant kernel).  `frac` counts
    the algorithmic pair flops times the k(k+1)/2 digit products of k planes
    (no tile padding); `frac_executed` the flops the tensor cores executed
    (every 128 x N tile in full, K padded to 64)."""
    peaks, peak_kind = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    achieved_exec = (pair_fl / (pair_ms / 1e3) / 1e12) if pair_ms > 0 else None
    prods = nslices * (nslices + 1) / 2
    achieved = (alg_flops * prods / (pair_ms / 1e3) / 1e12) if (pair_ms > 0 and alg_flops) else None
    tf = lambda q: (q[2] / (q[0] / 1e3) / 1e12) if q[0] > 0 else None  # noqa: E731
    return {"bound": "tensor", "kernel": "sliced_gemm_kernel (pair contraction, tcgen05 bf16 digit planes)",
            "achieved": achieved, "peak": peak, "peak_kind": f"bf16 dense sustained, {peak_kind}",
            "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
            "count": f"algorithmic pair flops (2 naux nv^2 per hole pair i <= j) x {prods:.0f} digit products",
            "achieved_executed": achieved_exec, "frac_executed": (achieved_exec / peak) if achieved_exec else None,
            "padding": (pair_fl / (alg_flops * prods)) if alg_flops else None,
            "traffic": traffic_per_launch(workload, pair_fl / max(pair_n, 1)) if pair_n else None,
            "traffic_note": "DRAM bytes per average pair launch: bytes per executed flop of one ncu capture of "
                            "a small pair launch, times this run's executed flops per launch",
            "launches": pair_n, "avg_launch_ms": pair_ms / max(pair_n, 1),
            "executed_flops_per_launch": pair_fl / max(pair_n, 1),
            "share_of_step": pair_ms / step_ms if step_ms > 0 else None,
            "syrk": {"ms": syrk[0], "launches": syrk[1], "tflops": tf(syrk)},
            "plain": {"ms": plain[0], "launches": plain[1], "tflops": tf(plain)}}


def batch_arm(args):
    """64 ragged instances per step through dsrg_fno_batch_run (autotuned
    worker count): E_vv, D_vv, NOs, the p_o cut and the correction of each."""
    import numpy as np
    import torch

    import paper_2312_07008_gb300 as pkg
    from synth.problems import batch_sizes, batch_problem

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    dev = torch.device("cuda", local)
    sizes = batch_sizes()
    probs = [batch_problem(k) for k in range(len(sizes))]
    n = len(probs)
    gps = [pkg.problem_from_synth(p, dev, pkg.SLICED_BF16, args.nslices) for p in probs]
    dvv = [torch.empty((p.nvir, p.nvir), dtype=torch.float64, device=dev) for p in probs]
    on = [torch.empty(p.nvir, dtype=torch.float64, device=dev) for p in probs]
    no = [torch.empty((p.nvir, p.nvir), dtype=torch.float64, device=dev) for p in probs]
    cut = (pkg.MODE_PO, BATCH_CUT, 0.01)

    def step(items):
        return pkg.dsrg_fno_batch_run(items, dvv, cut, on, no, correction=True, nworkers=0)

    for _ in range(args.warmup):
        step(gps)
    workers = pkg.dsrg_fno_batch_last_workers()
    stream = torch.cuda.current_stream()
    barrier()
    clk = ClockSampler(local, args.clock_ms)
    clk.start()
    time.sleep(0.3)
    # timed steps without the profiling hooks: eight workers recording events
    # under one lock distort the batch's wall time
    pkg.dsrg_fno_launch_count(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        res = step(gps)
    ev1.record(stream)
    barrier()
    launches = pkg.dsrg_fno_launch_count()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.stop()
    # the same steps again with the hooks on: kernel and phase breakdown
    pkg.dsrg_fno_profile_enable(True)
    for _ in range(args.steps):
        step(gps)
    barrier()
    pkg.dsrg_fno_profile_enable(False)
    q = {nm: pkg.dsrg_fno_profile_query(nm) for nm in ("sliced_gemm_pair", "sliced_gemm_syrk", "sliced_gemm_plain")}
    # stream time per step summed over the concurrent workers
    phases = {}
    for nm in PHASES:
        t_ms, n_l, _ = pkg.dsrg_fno_profile_query(nm)
        phases[nm] = {"stream_ms_per_step": t_ms / args.steps, "launches_or_calls": n_l}
    ms_max = max_over_ranks(ms, dist, dev)
    value = replica_rate(args.steps * n, world, ms_max)
    flops = sum(algorithmic_flops(p) for p in probs)

    # ---- end to end: every instance's inputs from pinned host memory each
    # step, into one of two device input sets on a copy stream: the copy of
    # batch i + 1 runs while batch i computes (the batch call returns only
    # when its instances are done, so the copy is issued just before it)
    host = []
    for p in probs:
        host.append({k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
                     for k, v in (("B", p.B), ("eps", p.eps), ("g1", p.gamma1), ("l2", p.lambda2))
                     if v is not None})
    sets, gsets = [], []
    for _ in range(2):
        dbufs = [{k: torch.empty_like(v, device=dev) for k, v in h.items()} for h in host]
        sets.append(dbufs)
        gsets.append([pkg.Problem(p.ncore, p.nact, p.nvir, p.naux, db["B"], db["eps"], db.get("g1"),
                                  db.get("l2"), None, p.weights, p.s, pkg.SLICED_BF16, args.nslices)
                      for p, db in zip(probs, dbufs)])
    h2d = sum(v.numel() * v.element_size() for h in host for v in h.values())
    on_host = [torch.empty(p.nvir, dtype=torch.float64).pin_memory() for p in probs]
    d2h = sum(x.numel() * 8 for x in on_host) + n * 8 * 3
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]

    def issue_copy(j):
        with torch.cuda.stream(copy_stream):
            for h, db in zip(host, sets[j]):
                for k in h:
                    db[k].copy_(h[k], non_blocking=True)
        copied[j].record(copy_stream)

    def e2e_run(nsteps):
        torch.cuda.synchronize()
        issue_copy(0)
        r = None
        for i in range(nsteps):
            j = i % 2
            copied[j].synchronize()  # this batch's inputs are on the device
            if i + 1 < nsteps:
                issue_copy(1 - j)  # set 1 - j was last read by batch i - 1, which has returned
            r = step(gsets[j])
            for a, b in zip(on_host, on):
                a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        return r

    e2e_run(1)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    barrier()
    e2e_value = replica_rate(args.steps * n, world, max_over_ranks(e0.elapsed_time(e1), dist, dev))

    # ---- the float64 GPU form on every 4th instance (a 16-instance sample)
    fp64 = None
    if args.fp64_steps > 0:
        idx = list(range(0, n, 4))
        g64 = [pkg.problem_from_synth(probs[i], dev, pkg.FP64) for i in idx]
        sub = lambda xs: [xs[i] for i in idx]  # noqa: E731
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        f0.record(stream)
        r64 = pkg.dsrg_fno_batch_run(g64, sub(dvv), cut, sub(on), sub(no), correction=True, nworkers=0)
        f1.record(stream)
        barrier()
        fms = f0.elapsed_time(f1)
        rf = pkg.dsrg_fno_batch_run(sub(gps), sub(dvv), cut, sub(on), sub(no), correction=True, nworkers=workers)
        fl64 = sum(algorithmic_flops(probs[i]) for i in idx)
        fp64 = {"sample": "every 4th instance (16)", "instances_per_s": len(idx) / (fms / 1e3),
                "gflops": fl64 / (fms / 1e3) / 1e9,
                "fast_minus_fp64": {"max_abs_e2": max(abs(a["e2"] - b["e2"]) for a, b in zip(rf, r64)),
                                    "max_abs_de": max(abs(a["de"] - b["de"]) for a, b in zip(rf, r64)),
                                    "nkept_equal": all(a["nkept"] == b["nkept"] for a, b in zip(rf, r64))}}

    alg = sum(pair_alg_flops(pp, [r["nkept"]]) for pp, r in zip(probs, res)) * args.steps
    roofline = roofline_of(*q["sliced_gemm_pair"], q["sliced_gemm_syrk"], q["sliced_gemm_plain"], ms,
                           alg_flops=alg, nslices=args.nslices)
    roofline["note"] = "kernel times from a second, profiled run of the same steps"
    line = {
        "metric": METRIC, "value": value, "unit": "instances/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"bf16 digit planes (k={args.nslices}) -> exact f32 level sums -> f64",
        "data": "synthetic",
        "config": batch_config(args.nslices),
        "workers": workers,
        "gflops": flops * value / n / 1e9,
        "s_per_step": ms_max / args.steps / 1e3,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "instances/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "phases": phases,
        "clocks": clocks,
        "fp64_form": fp64,
        "result": {"sum_e2": sum(r["e2"] for r in res), "sum_nkept": sum(r["nkept"] for r in res),
                   "sum_de": sum(r["de"] for r in res)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline([r["nkept"] for r in res])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
