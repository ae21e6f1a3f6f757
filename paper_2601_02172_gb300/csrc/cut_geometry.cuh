// Per-tet geometry of the X-FEM setup, shared by the setup kernels and a host-compiled check
// (the functions are __host__ __device__): classification of a tet against K level sets and
// the exact moments of the two sides of a cut tet.
#pragma once

#include <math.h>

#include "xfft_kernels.h"

#define XFFT_HD __host__ __device__

namespace xfft {

// Classification of tet (a, b, c, d vertex values per level set): returns the 2-bit code and,
// for a cut tet, the minus / plus phases; *two is set if a second interface cuts the tet.
XFFT_HD inline unsigned classify_tet(const double* const* Lv, int nL, int* pm, int* pp,
                                        bool* two) {
  int first = nL;
  bool cut = false;
  for (int l = 0; l < nL; ++l) {
    const double* x = Lv[l];
    const double mn = fmin(fmin(x[0], x[1]), fmin(x[2], x[3]));
    const double mx = fmax(fmax(x[0], x[1]), fmax(x[2], x[3]));
    if (first == nL) {
      if (mn < 0.0) {  // minus phase if any vertex is negative
        first = l;
        cut = mx > 0.0;
        *pp = nL;
      }
    } else if (cut && mn < 0.0) {
      if (mx > 0.0) *two = true;
      if (*pp == nL) *pp = l;
    }
  }
  *pm = first;
  return cut ? kCodeCut : phase_code(first);
}

// ---------------------------------------------------------------- side moments
struct Moments {
  double m[4];
  double M[10];
};

XFFT_HD inline double det4(const double b[4][4]) {
  // Laplace expansion along the first row
  double d = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int cols[3];
    int q = 0;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
      if (cc != c) cols[q++] = cc;
    const double m3 = b[1][cols[0]] * (b[2][cols[1]] * b[3][cols[2]] - b[2][cols[2]] * b[3][cols[1]])
                    - b[1][cols[1]] * (b[2][cols[0]] * b[3][cols[2]] - b[2][cols[2]] * b[3][cols[0]])
                    + b[1][cols[2]] * (b[2][cols[0]] * b[3][cols[1]] - b[2][cols[1]] * b[3][cols[0]]);
    d += ((c & 1) ? -1.0 : 1.0) * b[0][c] * m3;
  }
  return d;
}

// Add the moments of the sub-tetrahedron whose vertices have parent barycentric coordinates
// beta[v][.]: its volume is |det beta| |T|, int N_b = vol/4 sum_v beta_vb and
// int N_b N_c = vol/20 (sum_v beta_vb beta_vc + (sum_v beta_vb)(sum_v beta_vc)).
XFFT_HD inline void add_subtet(Moments& acc, const double b0[4], const double b1[4],
                                  const double b2[4], const double b3[4], double vol) {
  const double B[4][4] = {{b0[0], b0[1], b0[2], b0[3]},
                          {b1[0], b1[1], b1[2], b1[3]},
                          {b2[0], b2[1], b2[2], b2[3]},
                          {b3[0], b3[1], b3[2], b3[3]}};
  const double vs = fabs(det4(B)) * vol;
  double S[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) S[c] = B[0][c] + B[1][c] + B[2][c] + B[3][c];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc.m[c] += 0.25 * vs * S[c];
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int c = b; c < 4; ++c) {
      const double pp = B[0][b] * B[0][c] + B[1][b] * B[1][c] + B[2][b] * B[2][c] + B[3][b] * B[3][c];
      acc.M[midx(b, c)] += vs / 20.0 * (pp + S[b] * S[c]);
    }
}

XFFT_HD inline void unit_bary(int a, double out[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = (c == a) ? 1.0 : 0.0;
}

// barycentric point where L_h = 0 on the edge (a, b) (L_a L_b < 0), or vertex a if L_a = 0
XFFT_HD inline void edge_point(const double L[4], int a, int b, double out[4]) {
  if (L[a] == 0.0) {
    unit_bary(a, out);
    return;
  }
  const double t = L[a] / (L[a] - L[b]);
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = 0.0;
  out[a] = 1.0 - t;
  out[b] = t;
}

// Moments of side s (+1: s L_h >= 0) of a cut tet with nodal values L.
//   one strictly positive vertex a:   tet (a, edge points to the others)
//   one strictly negative vertex q:   prism (other three) -> (their edge points to q)
//   two and two:                       prism (a1, x11, x12) -> (a2, x21, x22)
XFFT_HD inline void side_moments(const double L[4], int s, double vol, Moments& out) {
#pragma unroll
  for (int c = 0; c < 4; ++c) out.m[c] = 0.0;
#pragma unroll
  for (int c = 0; c < 10; ++c) out.M[c] = 0.0;
  int P[4], Q[4], Z[4];
  int np = 0, nq = 0, nz = 0;
  for (int a = 0; a < 4; ++a) {
    const double x = s * L[a];
    if (x > 0.0)
      P[np++] = a;
    else if (x < 0.0)
      Q[nq++] = a;
    else
      Z[nz++] = a;
  }
  double v[6][4];
  if (np == 1) {
    const int a = P[0];
    unit_bary(a, v[0]);
    int k = 1;
    for (int i = 0; i < nq; ++i) edge_point(L, a, Q[i], v[k++]);
    for (int i = 0; i < nz; ++i) unit_bary(Z[i], v[k++]);
    add_subtet(out, v[0], v[1], v[2], v[3], vol);
  } else if (nq == 1) {
    const int q = Q[0];
    int k = 0;
    for (int a = 0; a < 4; ++a) {
      if (a == q) continue;
      unit_bary(a, v[k]);
      edge_point(L, a, q, v[3 + k]);
      ++k;
    }
    add_subtet(out, v[0], v[1], v[2], v[3], vol);
    add_subtet(out, v[1], v[2], v[3], v[4], vol);
    add_subtet(out, v[2], v[3], v[4], v[5], vol);
  } else {
    const int a1 = P[0], a2 = P[1], b1 = Q[0], b2 = Q[1];
    unit_bary(a1, v[0]);
    edge_point(L, a1, b1, v[1]);
    edge_point(L, a1, b2, v[2]);
    unit_bary(a2, v[3]);
    edge_point(L, a2, b1, v[4]);
    edge_point(L, a2, b2, v[5]);
    add_subtet(out, v[0], v[1], v[2], v[3], vol);
    add_subtet(out, v[1], v[2], v[3], v[4], vol);
    add_subtet(out, v[2], v[3], v[4], v[5], vol);
  }
}

}  // namespace xfft
