// Host build of the CUDA path's per-tet setup geometry (classification against K level sets and
// the exact side moments of a cut tet), for the CPU tests that compare it with the oracle.
// No kernels: every function called here is __host__ __device__.
#include "cut_geometry.cuh"

extern "C" {

// m[4] = int_side N_b, M[10] = int_side N_b N_c (packed 00,01,02,03,11,12,13,22,23,33)
void host_side_moments(const double* L, int s, double vol, double* m, double* M) {
  xfft::Moments mo;
  xfft::side_moments(L, s, vol, mo);
  for (int b = 0; b < 4; ++b) m[b] = mo.m[b];
  for (int k = 0; k < 10; ++k) M[k] = mo.M[k];
}

// Lv: nL x 4 vertex values; returns the 2-bit tet code, the side phases and the two-interface flag
unsigned host_classify_tet(const double* Lv, int nL, int* pm, int* pp, int* two) {
  const double* pv[xfft::kMaxPhases - 1];
  for (int l = 0; l < nL; ++l) pv[l] = Lv + 4 * l;
  bool t = false;
  *pm = 0;
  *pp = nL;
  const unsigned c = xfft::classify_tet(pv, nL, pm, pp, &t);
  *two = t ? 1 : 0;
  return c;
}

}  // extern "C"
