// Host replay of the element bodies of the full PT2 energy (csrc/mr_terms.cuh)
// for the CPU tests: the same per-element functions the GPU kernels loop over,
// run in stage order by plain host loops on a problem read from a binary file;
// prints the energy beyond E_vv.  Test infrastructure only (the library has no
// host path).  Input: int32 nc, na, nv, naux, has_f, has_l3; float64 s; B
// [naux][nh][np]; eps; f_hp [nh][np] if has_f; Gamma1; Lambda2; Lambda3 if has_l3.
#include <cmath>
using std::expm1;
using std::fma;
#include <cstdio>
#include <vector>

#include "../../paper_2312_07008_gb300/csrc/mr_terms.cuh"

using namespace dsrg;

static std::vector<double> read_doubles(FILE* f, long n) {
  std::vector<double> v(n);
  if (n > 0 && fread(v.data(), sizeof(double), n, f) != (size_t)n) v.clear();
  return v;
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int h[6];
  double s;
  if (fread(h, sizeof(int), 6, f) != 6 || fread(&s, sizeof(double), 1, f) != 1) return 2;
  const int nc = h[0], na = h[1], nv = h[2], nq = h[3], nh = nc + na, np = na + nv;
  auto B = read_doubles(f, (long)nq * nh * np);
  auto eps = read_doubles(f, nc + na + nv);
  auto fh = read_doubles(f, h[4] ? (long)nh * np : 0);
  auto g1 = read_doubles(f, (long)na * na);
  auto l2 = read_doubles(f, (long)na * na * na * na);
  auto l3 = read_doubles(f, h[5] ? (long)na * na * na * na * na * na : 0);
  fclose(f);
  const long n4 = (long)nh * nh * np * na, n4a = (long)na * nh * np * na, n1 = (long)nh * np;
  std::vector<double> nu(n4), tp(n4), xp(n4), z1(n4), z2(n4a), z3(n4a), g2t((long)nh * nh * na * na),
      w3((long)nh * na * na * na), t1(n1), x1(n1), tt1(n1), gt1((long)nh * na);
  // <ay|ij> = sum_Q B[Q][i][a] B[Q][j][y], the GEMM of the GPU path
  for (int i = 0; i < nh; ++i)
    for (int a = 0; a < np; ++a)
      for (int j = 0; j < nh; ++j)
        for (int y = 0; y < na; ++y) {
          double acc = 0.0;
          for (int q = 0; q < nq; ++q) acc += B[((long)q * nh + i) * np + a] * B[((long)q * nh + j) * np + y];
          nu[(((long)i * np + a) * nh + j) * na + y] = acc;
        }
  MRArgs A{};
  A.nc = nc;
  A.na = na;
  A.nv = nv;
  A.nh = nh;
  A.np = np;
  A.s = s;
  A.eps = eps.data();
  A.f_hp = h[4] ? fh.data() : nullptr;
  A.g1 = g1.data();
  A.l2 = l2.data();
  A.l3 = h[5] ? l3.data() : nullptr;
  A.nu = nu.data();
  A.tp = tp.data();
  A.xp = xp.data();
  A.t1 = t1.data();
  A.x1 = x1.data();
  A.z1 = z1.data();
  A.tpp = nu.data();
  A.z2 = z2.data();
  A.z3 = z3.data();
  A.g2t = g2t.data();
  A.w3 = w3.data();
  A.tt1 = tt1.data();
  A.gt1 = gt1.data();
  for (long i = 0; i < n4; ++i) mr_amp_elem(A, i);
  for (long i = 0; i < n1; ++i) mr_t1_elem(A, i);
  for (long i = 0; i < n4; ++i) mr_z1_elem(A, i);
  for (long i = 0; i < n4; ++i) mr_tpp_elem(A, i);
  for (long i = 0; i < n4a; ++i) mr_z23_elem(A, i);
  for (long i = 0; i < (long)nh * nh * na * na; ++i) mr_g2t_elem(A, i);
  for (long i = 0; i < (long)nh * na * na * na; ++i) mr_w3_elem(A, i);
  for (long i = 0; i < n1; ++i) mr_t1img_elem(A, i);
  double e = 0.0;
  for (long i = 0; i < n4; ++i) e += mr_energy_elem(A, i);
  for (long i = 0; i < n1; ++i) e += mr_energy1_elem(A, i);
  printf("%.17g\n", 2.0 * e);
  return 0;
}
