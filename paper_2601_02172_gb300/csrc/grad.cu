// Gradient of a scalar loss through the effective stiffness (not in the paper).
//
// The six converged load cases u_k (eps_bar = E_k, Mandel basis) are stationary points of the
// cell energy, and the X-FEM basis (including the scaling D0, built from grad^s only, eq.
// XFFT_diagonal) does not depend on C, so for any parameter theta of C
//   dC_kl / dtheta = (1/|Y|) int_Y eps_k : (dC/dtheta) : eps_l,   eps_k = E_k + grad^s u_k
// (the energy identity used in App. A).  With C = s_v (lambda_p I(x)I + 2 mu_p I_sym) and
// G = dLoss/dC_eff this gives, per tet or cut-tet side,
//   dL/dlambda_p += s_v sum_kl G_kl int tr eps_k tr eps_l / |Y|
//   dL/dmu_p     += s_v sum_kl G_kl int 2 eps_k : eps_l / |Y|
//   dL/ds_v      += sum_kl G_kl int eps_k : C_p : eps_l / |Y|
// and the energy form C_kl = int eps_k : C : eps_l / |Y| as a by-product.
//
// Arithmetic type T: double for the FP64 solver; float for the mixed-precision solver.  There the
// standard displacements are first split into float pairs u = hi + lo (hi = u rounded to FP32,
// lo = the rounded remainder); a node difference (hi_a - hi_b) + (lo_a - lo_b) then carries the
// FP64 difference to FP32 precision without FP64 arithmetic (hi_a - hi_b is exact for neighbours
// within a factor two of each other, and otherwise rounds relative to the difference itself).
// The enriched strains are still formed in FP64 (products with 1/sqrt(D0), then differences);
// strains and their products are FP32, each item's contribution accumulated in FP64.
#include <cuda_runtime.h>
#include <math.h>

#include "xfft_kernels.h"

namespace xfft {

// u = hi + lo in float pairs (hi = fl32(u), lo = fl32(u - hi))
__global__ void k_split_hilo(const double* __restrict__ u, float* __restrict__ hi, float* __restrict__ lo,
                             long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = u[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

// partial values: dlambda[p] (p < kMaxPhases), dmu[p], C_energy (21 upper entries)
constexpr int kNG = kGradValues;
constexpr int kNGC = 2 * kMaxPhases;  // first C_energy slot

__device__ __forceinline__ int upper_idx(int k, int l) {
  // k <= l, row-major upper triangle of 6x6
  return k * 6 - (k * (k - 1)) / 2 + (l - k);
}

__device__ __forceinline__ void unit_strain(int k, double (&e)[6]) {
  const double r = 0.70710678118654752440;
  for (int i = 0; i < 6; ++i) e[i] = 0.0;
  e[k] = k < 3 ? 1.0 : r;
}

template <typename T>
__device__ __forceinline__ T dd6(const T* a, const T* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + T(2) * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5]);
}

// One uncut tet t (compile time) of voxel v: strains of the six load cases, their pair products,
// the phase sums and the energy-form entries (accumulated in T per thread; FP32 sums of a few
// dozen items are exact to ~1e-7), and the voxel-scale contribution.
template <typename T, int t>
__device__ __forceinline__ void grad_uncut_tet(const double* __restrict__ U, const float* __restrict__ Uh,
                                               const float* __restrict__ Ul, const GradArgs& a,
                                               const T* Gk, long long v, int i3, int j3, int k3, int ph,
                                               T (&acc)[kNG], double& contrib) {
  const GridDev& g = a.g;
  constexpr int p = perm_p(t), q = perm_q(t), r = perm_r(t);
  long long nd[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) nd[c] = corner_node(g, i3, j3, k3, tet_corner(t, c));
  const T ih[3] = {(T)(1.0 / g.h[0]), (T)(1.0 / g.h[1]), (T)(1.0 / g.h[2])};
  const T rs = (T)0.70710678118654752440;
  T eps[6][6], tr[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    T H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      // the differences cancel: formed in FP64 (FP64 solver) or from the float pairs
      T d01, d12, d23;
      if constexpr (sizeof(T) == 8) {
        const double* uk = U + k * a.stride + i * g.N;
        const double u0 = uk[nd[0]], u1 = uk[nd[1]], u2 = uk[nd[2]], u3 = uk[nd[3]];
        d01 = u1 - u0;
        d12 = u2 - u1;
        d23 = u3 - u2;
      } else {
        const long long o = k * a.stride + i * g.N;
        const float h0 = Uh[o + nd[0]], h1 = Uh[o + nd[1]], h2 = Uh[o + nd[2]], h3 = Uh[o + nd[3]];
        const float l0 = Ul[o + nd[0]], l1 = Ul[o + nd[1]], l2 = Ul[o + nd[2]], l3 = Ul[o + nd[3]];
        d01 = (h1 - h0) + (l1 - l0);
        d12 = (h2 - h1) + (l2 - l1);
        d23 = (h3 - h2) + (l3 - l2);
      }
      H[i][p] = d01 * ih[p];
      H[i][q] = d12 * ih[q];
      H[i][r] = d23 * ih[r];
    }
    eps[k][0] = H[0][0];
    eps[k][1] = H[1][1];
    eps[k][2] = H[2][2];
    eps[k][3] = T(0.5) * (H[1][2] + H[2][1]);
    eps[k][4] = T(0.5) * (H[0][2] + H[2][0]);
    eps[k][5] = T(0.5) * (H[0][1] + H[1][0]);
    eps[k][k] += k < 3 ? T(1) : rs;  // unit Mandel strain E_k
    tr[k] = eps[k][0] + eps[k][1] + eps[k][2];
  }
  const T lam = (T)a.ph.lam[ph], mu = (T)a.ph.mu[ph];
  const double sv = a.scale ? (double)a.scale[v] : 1.0;
  const double w = g.vol_tet / g.volY;
  const T wsv = (T)(w * sv);
  T ql = T(0), qm = T(0);
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int l = k; l < 6; ++l) {
      const T tt = tr[k] * tr[l];
      const T ee = T(2) * dd6(eps[k], eps[l]);
      const T gk = Gk[upper_idx(k, l)];
      ql += gk * tt;
      qm += gk * ee;
      acc[kNGC + upper_idx(k, l)] += wsv * (lam * tt + mu * ee);
    }
  // per-phase sums with compile-time slots (no local-memory indexing)
  if (ph == 0) {
    acc[0] += wsv * ql;
    acc[kMaxPhases] += wsv * qm;
  } else if (ph == 1) {
    acc[1] += wsv * ql;
    acc[kMaxPhases + 1] += wsv * qm;
  } else {
    acc[2] += wsv * ql;
    acc[kMaxPhases + 2] += wsv * qm;
  }
  contrib = w * (double)(lam * ql + mu * qm);
}

// block: 32 voxels (x) by 6 tets (y); each warp handles one tet of 32 voxels
template <typename T>
__global__ void __launch_bounds__(192) k_grad_uncut(const double* __restrict__ U, const float* __restrict__ Uh,
                                                     const float* __restrict__ Ul, const GradArgs a,
                                                     double* __restrict__ dscale) {
  __shared__ double sds[6][32];
  __shared__ double red[kNG * 32];
  __shared__ T Gk[21];  // G_kl + G_lk (k < l), G_kk: the weights of the upper-triangle pair sums
  const int lane = threadIdx.x, t = threadIdx.y;
  const int tid = lane + 32 * t;
  if (tid < 36) {
    const int k = tid / 6, l = tid - 6 * (tid / 6);
    if (k <= l) Gk[upper_idx(k, l)] = (T)(k == l ? a.G[k * 6 + l] : a.G[k * 6 + l] + a.G[l * 6 + k]);
  }
  __syncthreads();
  const GridDev& g = a.g;
  T acc[kNG];
#pragma unroll
  for (int i = 0; i < kNG; ++i) acc[i] = T(0);
  const long long ngroups = (g.N + 31) / 32;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long long v = grp * 32 + lane;
    double contrib = 0.0;
    if (v < g.N) {
      const unsigned cd = (a.code[v] >> (2 * t)) & 3u;
      if (cd != kCodeCut) {
        const int ph = code_phase(cd);
        // voxel coordinates (32-bit division where the grid allows it)
        int i3, j3, k3;
        if (g.N <= 0xffffffffLL) {
          const unsigned vu = (unsigned)v, r2 = vu / (unsigned)g.n2;
          k3 = (int)(vu - r2 * (unsigned)g.n2);
          i3 = (int)(r2 / (unsigned)g.n1);
          j3 = (int)(r2 - (unsigned)i3 * (unsigned)g.n1);
        } else {
          k3 = (int)(v % g.n2);
          j3 = (int)((v / g.n2) % g.n1);
          i3 = (int)(v / ((long long)g.n1 * g.n2));
        }
        switch (t) {  // uniform per warp
          case 0: grad_uncut_tet<T, 0>(U, Uh, Ul, a, Gk, v, i3, j3, k3, ph, acc, contrib); break;
          case 1: grad_uncut_tet<T, 1>(U, Uh, Ul, a, Gk, v, i3, j3, k3, ph, acc, contrib); break;
          case 2: grad_uncut_tet<T, 2>(U, Uh, Ul, a, Gk, v, i3, j3, k3, ph, acc, contrib); break;
          case 3: grad_uncut_tet<T, 3>(U, Uh, Ul, a, Gk, v, i3, j3, k3, ph, acc, contrib); break;
          case 4: grad_uncut_tet<T, 4>(U, Uh, Ul, a, Gk, v, i3, j3, k3, ph, acc, contrib); break;
          default: grad_uncut_tet<T, 5>(U, Uh, Ul, a, Gk, v, i3, j3, k3, ph, acc, contrib); break;
        }
      }
    }
    sds[t][lane] = contrib;
    __syncthreads();
    if (t == 0 && v < g.N)
      dscale[v] = sds[0][lane] + sds[1][lane] + sds[2][lane] + sds[3][lane] + sds[4][lane] + sds[5][lane];
    __syncthreads();
  }
  double accd[kNG], tot[kNG];
#pragma unroll
  for (int i = 0; i < kNG; ++i) accd[i] = (double)acc[i];
  block_sum<kNG>(accd, red, tot);
  if (tid == 0)
    for (int i = 0; i < kNG; ++i) a.partials[(long long)i * a.nparts + blockIdx.x] = tot[i];
}

template <typename T>
__global__ void __launch_bounds__(64) k_grad_cut(const double* __restrict__ U, const float* __restrict__ Uh,
                                                  const float* __restrict__ Ul,
                                                  const double* __restrict__ isD, const CutData cd,
                                                  const GradArgs a, double* __restrict__ dscale) {
  __shared__ double red[kNG * 32];
  __shared__ T Gk[21];  // G_kl + G_lk (k < l), G_kk
  if (threadIdx.x < 36) {
    const int k = threadIdx.x / 6, l = threadIdx.x - 6 * (threadIdx.x / 6);
    if (k <= l) Gk[upper_idx(k, l)] = (T)(k == l ? a.G[k * 6 + l] : a.G[k * 6 + l] + a.G[l * 6 + k]);
  }
  __syncthreads();
  const GridDev& g = a.g;
  const long long N = g.N;
  const int nX = a.nX, ncut = cd.ncut;
  const double inv = 1.0 / g.volY;
  double ih[3];
  for (int k = 0; k < 3; ++k) ih[k] = 1.0 / g.h[k];
  double acc[kNG];
#pragma unroll
  for (int i = 0; i < kNG; ++i) acc[i] = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncut; e += gridDim.x * blockDim.x) {
    int nd[4], ei[4];
    for (int k = 0; k < 4; ++k) {
      nd[k] = cd.ip[k * ncut + e];
      ei[k] = cd.ip[(4 + k) * ncut + e];
    }
    const int vox = cd.ip[8 * ncut + e];
    const int t = cd.ip[9 * ncut + e];
    const int sph = cd.ip[kCutFieldPhases * ncut + e];
    double gr[4][3];
    tet_grads<double>(t, ih, gr);
    double L[4];
    for (int b = 0; b < 4; ++b) L[b] = cd.dp[(long long)cut_f_L(b) * ncut + e];
    const double sv = a.scale ? (double)a.scale[vox] : 1.0;
    double contrib = 0.0;
    for (int si = 0; si < 2; ++si) {
      const double s = si == 0 ? 1.0 : -1.0;
      const int ph = si == 0 ? cut_phase_plus(sph) : cut_phase_minus(sph);
      const double lam = a.ph.lam[ph], mu = a.ph.mu[ph];
      double c[4], gam[3] = {0, 0, 0};
      for (int b = 0; b < 4; ++b) {
        c[b] = fabs(L[b]) - s * L[b];
        for (int x = 0; x < 3; ++x) gam[x] += c[b] * gr[b][x];
      }
      T M[10];
      for (int k = 0; k < 10; ++k) M[k] = (T)cd.dp[(long long)cut_f_M(si, k) * ncut + e];
      T Eb[6][4][6];  // [load case][b][component]
      T trb[6][4];
      if constexpr (sizeof(T) == 4) {
        // standard strain from the float pairs along the tet's path 0 -> e_p -> e_p+e_q -> (1,1,1);
        // enriched strain from FP64 differences of the physical enriched coefficients
        const int p = perm_p(t), q = perm_q(t), r = perm_r(t);
        const float ihf[3] = {(float)ih[0], (float)ih[1], (float)ih[2]};
        float cf[4], gamf[3];
        for (int b = 0; b < 4; ++b) cf[b] = (float)c[b];
        for (int x = 0; x < 3; ++x) gamf[x] = (float)gam[x];
        for (int k = 0; k < 6; ++k) {
          float Hs[3][3], Hw[3][3], wsf[4][3];
          for (int i = 0; i < 3; ++i) {
            const long long o = k * a.stride + i * N;
            float hv[4], lv[4];
            double wv[4];
            for (int aa = 0; aa < 4; ++aa) {
              hv[aa] = Uh[o + nd[aa]];
              lv[aa] = Ul[o + nd[aa]];
              const long long oe = (long long)i * nX + ei[aa];
              wv[aa] = U[k * a.stride + 3 * N + oe] * isD[oe];
              wsf[aa][i] = (float)wv[aa];
            }
            Hs[i][p] = ((hv[1] - hv[0]) + (lv[1] - lv[0])) * ihf[p];
            Hs[i][q] = ((hv[2] - hv[1]) + (lv[2] - lv[1])) * ihf[q];
            Hs[i][r] = ((hv[3] - hv[2]) + (lv[3] - lv[2])) * ihf[r];
            Hw[i][p] = (float)(wv[1] - wv[0]) * ihf[p];
            Hw[i][q] = (float)(wv[2] - wv[1]) * ihf[q];
            Hw[i][r] = (float)(wv[3] - wv[2]) * ihf[r];
          }
          const float rs = 0.70710678118654752440f;
          float es[6] = {Hs[0][0], Hs[1][1], Hs[2][2], 0.5f * (Hs[1][2] + Hs[2][1]),
                         0.5f * (Hs[0][2] + Hs[2][0]), 0.5f * (Hs[0][1] + Hs[1][0])};
          es[k] += k < 3 ? 1.0f : rs;  // unit Mandel strain E_k
          const float ew[6] = {Hw[0][0], Hw[1][1], Hw[2][2], 0.5f * (Hw[1][2] + Hw[2][1]),
                               0.5f * (Hw[0][2] + Hw[2][0]), 0.5f * (Hw[0][1] + Hw[1][0])};
          for (int b = 0; b < 4; ++b) {
            const float* wb = wsf[b];
            const float sw[6] = {wb[0] * gamf[0], wb[1] * gamf[1], wb[2] * gamf[2],
                                 0.5f * (wb[1] * gamf[2] + wb[2] * gamf[1]),
                                 0.5f * (wb[0] * gamf[2] + wb[2] * gamf[0]),
                                 0.5f * (wb[0] * gamf[1] + wb[1] * gamf[0])};
            for (int x = 0; x < 6; ++x) Eb[k][b][x] = es[x] + cf[b] * ew[x] + sw[x];
            trb[k][b] = Eb[k][b][0] + Eb[k][b][1] + Eb[k][b][2];
          }
        }
      } else
      for (int k = 0; k < 6; ++k) {
        const double* uk = U + k * a.stride;
        double us[4][3], ws[4][3];
        for (int aa = 0; aa < 4; ++aa)
          for (int x = 0; x < 3; ++x) {
            us[aa][x] = uk[x * N + nd[aa]];
            ws[aa][x] = uk[3 * N + (long long)x * nX + ei[aa]] * isD[(long long)x * nX + ei[aa]];
          }
        double Hs[3][3], Hw[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            Hs[i][j] = 0.0;
            Hw[i][j] = 0.0;
            for (int aa = 0; aa < 4; ++aa) {
              Hs[i][j] += us[aa][i] * gr[aa][j];
              Hw[i][j] += ws[aa][i] * gr[aa][j];
            }
          }
        double E[6];
        unit_strain(k, E);
        const double es[6] = {Hs[0][0] + E[0], Hs[1][1] + E[1], Hs[2][2] + E[2],
                              0.5 * (Hs[1][2] + Hs[2][1]) + E[3], 0.5 * (Hs[0][2] + Hs[2][0]) + E[4],
                              0.5 * (Hs[0][1] + Hs[1][0]) + E[5]};
        const double ew[6] = {Hw[0][0], Hw[1][1], Hw[2][2], 0.5 * (Hw[1][2] + Hw[2][1]),
                              0.5 * (Hw[0][2] + Hw[2][0]), 0.5 * (Hw[0][1] + Hw[1][0])};
        for (int b = 0; b < 4; ++b) {
          const double* wb = ws[b];
          const double sw[6] = {wb[0] * gam[0], wb[1] * gam[1], wb[2] * gam[2],
                                0.5 * (wb[1] * gam[2] + wb[2] * gam[1]),
                                0.5 * (wb[0] * gam[2] + wb[2] * gam[0]),
                                0.5 * (wb[0] * gam[1] + wb[1] * gam[0])};
          for (int x = 0; x < 6; ++x) Eb[k][b][x] = (T)(es[x] + c[b] * ew[x] + sw[x]);
          trb[k][b] = Eb[k][b][0] + Eb[k][b][1] + Eb[k][b][2];
        }
      }
      T ql = T(0), qm = T(0);
      const T lamT = (T)lam, muT = (T)mu;
#pragma unroll 1
      for (int l = 0; l < 6; ++l) {
        // the side's moment matrix applied to load case l's corner strains and traces, so that
        // each pair (k, l) costs one pass over load case k's corners
        T ME[4][6], mt[4];
        for (int b = 0; b < 4; ++b) {
          mt[b] = T(0);
          for (int x = 0; x < 6; ++x) ME[b][x] = T(0);
          for (int cc = 0; cc < 4; ++cc) {
            const T m = M[midx(b, cc)];
            mt[b] += m * trb[l][cc];
            for (int x = 0; x < 6; ++x) ME[b][x] += m * Eb[l][cc][x];
          }
        }
        for (int k = 0; k <= l; ++k) {
          T tt = T(0), ee = T(0);
          for (int b = 0; b < 4; ++b) {
            tt += trb[k][b] * mt[b];
            ee += dd6(Eb[k][b], ME[b]);
          }
          ee *= T(2);
          const T gk = Gk[upper_idx(k, l)];
          ql += gk * tt;
          qm += gk * ee;
          acc[kNGC + upper_idx(k, l)] += inv * sv * (double)(lamT * tt + muT * ee);
        }
      }
      acc[ph] += inv * sv * (double)ql;
      acc[kMaxPhases + ph] += inv * sv * (double)qm;
      contrib += inv * (double)(lamT * ql + muT * qm);
    }
    atomicAdd(&dscale[vox], contrib);
  }
  double tot[kNG];
  block_sum<kNG>(acc, red, tot);
  if (threadIdx.x == 0)
    for (int i = 0; i < kNG; ++i)
      a.partials[(long long)i * a.nparts + a.part_offset_cut + blockIdx.x] = tot[i];
}

int grad_blocks_uncut(const GridDev& g) {
  const long long ngroups = (g.N + 31) / 32;
  return (int)(ngroups < 4096 ? ngroups : 4096);
}
int grad_blocks_cut(int ncut) {
  const int nb = (ncut + 63) / 64;
  return nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
}

cudaError_t launch_grad(const double* U, const double* isD, CutData cd, const GradArgs& a,
                        double* dscale, float* hi, float* lo, cudaStream_t s) {
  const bool fp32 = hi != nullptr;
  if (fp32) {
    const long long n = 6 * a.stride;
    const long long nb = (n + 255) / 256;
    k_split_hilo<<<(int)(nb < 8192 ? nb : 8192), 256, 0, s>>>(U, hi, lo, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_grad_uncut<float><<<grad_blocks_uncut(a.g), dim3(32, 6), 0, s>>>(U, hi, lo, a, dscale);
  } else {
    k_grad_uncut<double><<<grad_blocks_uncut(a.g), dim3(32, 6), 0, s>>>(U, nullptr, nullptr, a, dscale);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fp32)
    k_grad_cut<float><<<grad_blocks_cut(cd.ncut), 64, 0, s>>>(U, hi, lo, isD, cd, a, dscale);
  else
    k_grad_cut<double><<<grad_blocks_cut(cd.ncut), 64, 0, s>>>(U, nullptr, nullptr, isD, cd, a, dscale);
  return cudaGetLastError();
}

__global__ void k_reduce_partials(const double* __restrict__ partials, int nparts, int ncount,
                                  double* __restrict__ out) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < ncount; i += blockDim.x) v += partials[(long long)k * nparts + i];
  double vv[1] = {v}, tot[1];
  block_sum<1>(vv, red, tot);
  if (threadIdx.x == 0) out[k] = tot[0];
}

// out[k] = sum_{i < ncount} partials[k * nparts + i] for k < nvals
cudaError_t launch_reduce_partials(const double* partials, int nvals, int nparts, int ncount,
                                   double* out, cudaStream_t s) {
  k_reduce_partials<<<nvals, 256, 0, s>>>(partials, nparts, ncount, out);
  return cudaGetLastError();
}

}  // namespace xfft
