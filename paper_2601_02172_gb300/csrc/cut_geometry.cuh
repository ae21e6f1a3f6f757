// Per-tet geometry of the X-FEM setup, shared by the setup kernels and a host-compiled check
// (the functions are __host__ __device__): classification of a tet against K level sets, the
// exact moments of the two sides of a cut tet, and the cut tet's scaled element matrix formed
// from them (the optional cache of the FP32 iterations).
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

// ---------------------------------------------------------------- cached element matrices
// The paper's caching strategy (Sec. 2.3, next to Algorithm 1): the scaled element matrix of
// every cut tet is formed once per microstructure instead of once per iteration.  On side s
// the strain at the parent P1 function N_b is E_b = es + c_b ew + sym(w_b (x) gamma) (see the
// apply kernels), so with the side moments M_bc = int N_b N_c every entry is a sum of
//   beta(x, u; y, v) = sym(e_x (x) u) : C : sym(e_y (x) v)
//                    = lambda u_x v_y + mu (delta_xy u.v + u_y v_x)
// over u, v in {grad N_a, gamma} with the weights (per side)
//   std (a,x)  - std (b,y):  V beta(x, g_a; y, g_b),  V = sum_bc M_bc
//   std (a,x)  - enr (b,y):  d_by [P beta(x, g_a; y, g_b) + m_b beta(x, g_a; y, gamma)]
//   enr (a,x)  - enr (b,y):  d_ax d_by [Q beta(x, g_a; y, g_b) + R_b beta(x, g_a; y, gamma)
//                                        + R_a beta(x, gamma; y, g_b) + M_ab beta(x, gamma; y, gamma)]
// with m_b = sum_c M_bc, R_a = sum_c M_ac c_c, P = sum_b m_b c_b, Q = sum_bc c_b M_bc c_c and
// d = D0^-1/2 of the enriched DOF.  Computed in FP64, stored as FP32: the upper triangle of the
// 24 x 24 matrix (local DOFs std 3a + x, then enr 12 + 3a + x) row by row, kCutPacked values
// per cut tet, structure of arrays kc[k * ncut + e].
XFFT_HD inline double beta_iso(int x, const double* u, int y, const double* v, double lam,
                                           double mu) {
  const double uv = x == y ? u[0] * v[0] + u[1] * v[1] + u[2] * v[2] : 0.0;
  return lam * u[x] * v[y] + mu * (uv + u[y] * v[x]);
}

struct SideW {
  double lam, mu, V, P, Q, m[4], R[4], M[4][4], gam[3];
};

// Per-side weights of a cut tet: the side's Lame constants, gamma = sum_b c_b grad N_b with
// c_b = |L_b| - s L_b, the moments M_bc (packed as cut_f_M) and their sums V, m_b, R_b, P, Q.
XFFT_HD inline void side_weights(const double L[4], double sgn, const double gr[4][3], const double Mp[10],
                                 double lam, double mu, SideW& W) {
  W.lam = lam;
  W.mu = mu;
  double c[4];
  for (int b = 0; b < 4; ++b) c[b] = fabs(L[b]) - sgn * L[b];
  for (int x = 0; x < 3; ++x) W.gam[x] = c[0] * gr[0][x] + c[1] * gr[1][x] + c[2] * gr[2][x] + c[3] * gr[3][x];
  for (int b = 0; b < 4; ++b)
    for (int cc = 0; cc < 4; ++cc) W.M[b][cc] = Mp[midx(b, cc)];
  W.V = W.P = W.Q = 0.0;
  for (int b = 0; b < 4; ++b) {
    W.m[b] = W.M[b][0] + W.M[b][1] + W.M[b][2] + W.M[b][3];
    W.R[b] = W.M[b][0] * c[0] + W.M[b][1] * c[1] + W.M[b][2] * c[2] + W.M[b][3] * c[3];
    W.V += W.m[b];
    W.P += W.m[b] * c[b];
    W.Q += W.R[b] * c[b];
  }
}

// Entry (i, j) of the scaled 24 x 24 element matrix (local DOFs std 3a + x, enr 12 + 3a + x),
// summed over the two sides; dsc = D0^-1/2 of the tet's enriched DOFs.
XFFT_HD inline double cut_element_entry(int i, int j, const SideW w[2], const double gr[4][3],
                                        const double dsc[4][3]) {
  if (j < i) {
    const int tmp = i;
    i = j;
    j = tmp;
  }
  const bool ie = i >= 12, je = j >= 12;
  const int a = (ie ? i - 12 : i) / 3, x = (ie ? i - 12 : i) % 3;
  const int b = (je ? j - 12 : j) / 3, y = (je ? j - 12 : j) % 3;
  double v = 0.0;
  for (int si = 0; si < 2; ++si) {
    const SideW& W = w[si];
    const double bgg = beta_iso(x, gr[a], y, gr[b], W.lam, W.mu);
    if (!je) {
      v += W.V * bgg;
    } else if (!ie) {
      v += dsc[b][y] * (W.P * bgg + W.m[b] * beta_iso(x, gr[a], y, W.gam, W.lam, W.mu));
    } else {
      v += dsc[a][x] * dsc[b][y] *
           (W.Q * bgg + W.R[b] * beta_iso(x, gr[a], y, W.gam, W.lam, W.mu) +
            W.R[a] * beta_iso(x, W.gam, y, gr[b], W.lam, W.mu) + W.M[a][b] * beta_iso(x, W.gam, y, W.gam, W.lam, W.mu));
    }
  }
  return v;
}

// Contributions of one cut tet to the enriched scaling (eq. XFFT_diagonal, per DOF) and, if
// want_off, to the off-diagonal entries of the per-node 3 x 3 Gram blocks.  On side s,
// grad N_X^a = sum_b N_b V_ab with V_ab = c_b g_a + delta_ab gamma, so
//   D_{a,k} = 1/2 sum_bc M_bc (V_ab . V_ac + V_ab[k] V_ac[k])
// and the (k, l) block entry is 1/2 sum_bc M_bc V_ab[k] V_ac[l] for k != l.  Mp[0] / Mp[1]: the
// packed moments of the plus / minus side; off[a] = entries (0,1), (0,2), (1,2).
XFFT_HD inline void cut_scaling_terms(const double L[4], const double gr[4][3], const double Mp[2][10],
                                      double acc[4][3], double off[4][3], bool want_off) {
  for (int a = 0; a < 4; ++a)
    for (int x = 0; x < 3; ++x) acc[a][x] = off[a][x] = 0.0;
  for (int si = 0; si < 2; ++si) {
    const double s = si == 0 ? 1.0 : -1.0;
    double c[4], gam[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 4; ++b) {
      c[b] = fabs(L[b]) - s * L[b];
      for (int x = 0; x < 3; ++x) gam[x] += c[b] * gr[b][x];
    }
    const double* M = Mp[si];
    for (int a = 0; a < 4; ++a) {
      double V[4][3];
      for (int b = 0; b < 4; ++b)
        for (int x = 0; x < 3; ++x) V[b][x] = c[b] * gr[a][x] + (a == b ? gam[x] : 0.0);
      for (int b = 0; b < 4; ++b)
        for (int cc = 0; cc < 4; ++cc) {
          const double w = M[midx(b, cc)];
          const double dot = V[b][0] * V[cc][0] + V[b][1] * V[cc][1] + V[b][2] * V[cc][2];
          for (int x = 0; x < 3; ++x) acc[a][x] += 0.5 * w * (dot + V[b][x] * V[cc][x]);
          if (want_off) {
            off[a][0] += 0.5 * w * V[b][0] * V[cc][1];
            off[a][1] += 0.5 * w * V[b][0] * V[cc][2];
            off[a][2] += 0.5 * w * V[b][1] * V[cc][2];
          }
        }
    }
  }
}

// Inverse of the symmetric positive definite 3 x 3 matrix (a00, a11, a22; a10, a20, a21) by its
// Cholesky factor: v = (inv00, inv11, inv22, inv10, inv20, inv21); false (and v = identity) on a
// non-positive pivot.
XFFT_HD inline bool block_inverse3(double a00, double a11, double a22, double a10, double a20, double a21,
                                   double v[6]) {
  v[0] = v[1] = v[2] = 1.0;
  v[3] = v[4] = v[5] = 0.0;
  if (!(a00 > 0.0)) return false;
  const double l00 = sqrt(a00);
  const double l10 = a10 / l00, l20 = a20 / l00;
  const double p11 = a11 - l10 * l10;
  if (!(p11 > 0.0)) return false;
  const double l11 = sqrt(p11);
  const double l21 = (a21 - l20 * l10) / l11;
  const double p22 = a22 - l20 * l20 - l21 * l21;
  if (!(p22 > 0.0)) return false;
  const double l22 = sqrt(p22);
  const double m00 = 1.0 / l00, m11 = 1.0 / l11, m22 = 1.0 / l22;
  const double m10 = -l10 * m00 * m11;
  const double m21 = -l21 * m11 * m22;
  const double m20 = -(l20 * m00 + l21 * m10) * m22;
  v[0] = m00 * m00 + m10 * m10 + m20 * m20;
  v[1] = m11 * m11 + m21 * m21;
  v[2] = m22 * m22;
  v[3] = m10 * m11 + m20 * m21;
  v[4] = m20 * m22;
  v[5] = m21 * m22;
  return true;
}

}  // namespace xfft
