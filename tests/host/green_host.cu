// Host build of the CUDA path's per-frequency Green solve (the 3x3 complex Cholesky factor of
// M(xi) in closed form and the two triangular solves), for the CPU test against the oracle.
#include "fft_fast.cuh"

namespace {
template <typename C, typename T>
int solve(const double* e, const double* s, const double* ih, double halfvol, double* F) {
  C ee[3], ss[3], f[3];
  for (int a = 0; a < 3; ++a) {
    ee[a].x = (T)e[2 * a];
    ee[a].y = (T)e[2 * a + 1];
    ss[a].x = (T)s[2 * a];
    ss[a].y = (T)s[2 * a + 1];
    f[a].x = (T)F[2 * a];
    f[a].y = (T)F[2 * a + 1];
  }
  xfft::fast::GreenFactor<C, T> gf;
  if (!xfft::fast::green_factor<C, T>(gf, ee[0], ee[1], ee[2], ss[0], ss[1], ss[2], (T)ih[0], (T)ih[1],
                                      (T)ih[2], (T)halfvol))
    return 0;
  xfft::fast::green_solve<C, T>(gf, f[0], f[1], f[2]);
  for (int a = 0; a < 3; ++a) {
    F[2 * a] = (double)f[a].x;
    F[2 * a + 1] = (double)f[a].y;
  }
  return 1;
}
}  // namespace

extern "C" int host_green_solve(int dbl, const double* e, const double* s, const double* ih, double halfvol,
                                double* F) {
  return dbl ? solve<double2, double>(e, s, ih, halfvol, F) : solve<float2, float>(e, s, ih, halfvol, F);
}
