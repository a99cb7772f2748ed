"""The particle-particle ladder of Eq. 6 on the GPU (dsrg_fno_ladder) against
the oracle's plain definition (4-index integrals formed explicitly), in both
arithmetic forms, on sizes that span several 128 x 48 tiles and ragged tails
of every contraction."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402


def inputs(nv, naux, npairs, seed):
    rng = np.random.default_rng(seed)
    Bv = 0.05 * rng.standard_normal((naux, nv, nv))
    Bv = (Bv + Bv.transpose(0, 2, 1)) / np.sqrt(2.0)   # (ac|..) factors are symmetric in a, c
    T = 0.01 * rng.standard_normal((npairs, nv, nv))
    return Bv, T


@pytest.mark.parametrize("prec", [pkg.FP64, pkg.SLICED_BF16], ids=["fp64", "fast"])
@pytest.mark.parametrize("nv,naux,npairs", [(37, 90, 11), (61, 200, 130), (9, 7, 3)])
def test_ladder_matches_oracle(prec, nv, naux, npairs):
    Bv, T = inputs(nv, naux, npairs, seed=nv + naux)
    ref = O.ladder(Bv, T)
    C = torch.empty((npairs, nv, nv), dtype=torch.float64, device="cuda")
    pkg.dsrg_fno_ladder(torch.from_numpy(Bv).cuda(), torch.from_numpy(T).cuda(), C, prec)
    got = C.cpu().numpy()
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"nv {nv} naux {naux} pairs {npairs} prec {prec}: max rel err {err:.2e}")
    assert err <= (1e-12 if prec == pkg.FP64 else 1e-10)


def test_ladder_rejects_non_finite_input():
    Bv, T = inputs(12, 20, 3, seed=5)
    T[1, 2, 3] = np.inf
    C = torch.empty((3, 12, 12), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DsrgFnoError) as ei:
        pkg.dsrg_fno_ladder(torch.from_numpy(Bv).cuda(), torch.from_numpy(T).cuda(), C)
    assert ei.value.status == -6
