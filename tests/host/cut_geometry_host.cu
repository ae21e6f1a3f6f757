// Host build of the CUDA path's per-tet setup geometry (classification against K level sets, the
// exact side moments of a cut tet and its scaled element matrix), for the CPU tests that compare
// it with the oracle.
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

// Scaled element matrix of a cut tet of type t (grid spacing h): packed upper triangle, 300
// values; Mplus / Mminus: packed side moments; dsc: D0^-1/2 (4 x 3); lame: lambda, mu of the
// plus side, then of the minus side (voxel scale included)
void host_cut_element_matrix(const double* L, int t, const double* h, const double* Mplus,
                             const double* Mminus, const double* dsc, const double* lame, double* K) {
  const double ih[3] = {1.0 / h[0], 1.0 / h[1], 1.0 / h[2]};
  double gr[4][3], d[4][3];
  xfft::tet_grads<double>(t, ih, gr);
  for (int a = 0; a < 4; ++a)
    for (int x = 0; x < 3; ++x) d[a][x] = dsc[3 * a + x];
  xfft::SideW w[2];
  xfft::side_weights(L, 1.0, gr, Mplus, lame[0], lame[1], w[0]);
  xfft::side_weights(L, -1.0, gr, Mminus, lame[2], lame[3], w[1]);
  int k = 0;
  for (int i = 0; i < 24; ++i)
    for (int j = i; j < 24; ++j) K[k++] = xfft::cut_element_entry(i, j, w, gr, d);
}

// One cut tet's contributions to D0 (acc, 4 x 3) and to the off-diagonal Gram entries (off,
// 4 x 3: (0,1), (0,2), (1,2)); Mplus / Mminus: packed side moments
void host_cut_scaling(const double* L, int t, const double* h, const double* Mplus, const double* Mminus,
                      double* acc, double* off) {
  const double ih[3] = {1.0 / h[0], 1.0 / h[1], 1.0 / h[2]};
  double gr[4][3], Mp[2][10], A[4][3], O[4][3];
  xfft::tet_grads<double>(t, ih, gr);
  for (int k = 0; k < 10; ++k) {
    Mp[0][k] = Mplus[k];
    Mp[1][k] = Mminus[k];
  }
  xfft::cut_scaling_terms(L, gr, Mp, A, O, true);
  for (int a = 0; a < 4; ++a)
    for (int x = 0; x < 3; ++x) {
      acc[3 * a + x] = A[a][x];
      off[3 * a + x] = O[a][x];
    }
}

// a = (a00, a11, a22, a10, a20, a21) -> v = the inverse in the same order; returns 1 if SPD
int host_block_inverse(const double* a, double* v) {
  return xfft::block_inverse3(a[0], a[1], a[2], a[3], a[4], a[5], v) ? 1 : 0;
}

}  // extern "C"
