// Stiffness apply launchers and the per-voxel average stress; the kernels are in
// apply_kernels.cuh.  This unit instantiates the one-interface kernels (two phases);
// apply_multi.cu instantiates those of two interfaces (three phases).
#include "apply_kernels.cuh"
#include "apply_cut.cuh"

namespace xfft {

XFFT_APPLY_INST_NPH(extern, float, 3)
XFFT_APPLY_INST_NPH(extern, double, 3)
XFFT_APPLY_INST_NPH(extern, dw, 3)

int apply_uncut_blocks(const GridDev& g) {
  const int gz = (g.n2 + kTZ - 2) / (kTZ - 1);
  const int gy = (g.n1 + kTY - 2) / (kTY - 1);
  const int gx = (g.n0 + kCX - 1) / kCX;
  return gz * gy * gx;
}

#ifndef XFFT_CUT_WAVES
#define XFFT_CUT_WAVES 2
#endif
constexpr int kCutBlocksMax = XFFT_CUT_WAVES * 4 * 152;  // waves of four resident blocks per SM
int apply_cut_blocks(int ncut) {
  const int nb = (ncut + kCutThreads - 1) / kCutThreads;
  return nb < 1 ? 1 : (nb > kCutBlocksMax ? kCutBlocksMax : nb);
}

constexpr int kCutBlocksTuneMax = 4 * 4 * 152;  // four waves of four resident blocks per SM
int apply_cut_blocks_max(int ncut) {
  const int nb = (ncut + kCutThreads - 1) / kCutThreads;
  const int cap = nb < kCutBlocksTuneMax ? nb : kCutBlocksTuneMax;
  const int def = apply_cut_blocks(ncut);
  return cap > def ? cap : def;
}

template <typename T>
cudaError_t launch_apply_uncut(const typename Store<T>::type* d, typename Store<T>::type* q,
                               const ApplyArgs& a, int n_rhs, cudaStream_t s) {
  return a.ph.nph > 2 ? launch_uncut_nph<T, 3>(d, q, a, n_rhs, s) : launch_uncut_nph<T, 2>(d, q, a, n_rhs, s);
}

// ---------------------------------------------------------------- cut tets from cached matrices
// FP32 cut-tet apply with the cached scaled element matrices (setup.cu, k_cut_matrix) for the
// applies of the inner CG iterations (no eps_bar, no stress integrals): q_e = K_e d_e on the
// local DOFs (std 3a + x, scaled enr 12 + 3a + x; the D0^-1/2 scaling is inside K_e).
// A block takes 32 cut tets at a time (threadIdx.x) for nr right-hand sides (threadIdx.y):
// the group's 32 packed matrices are staged in shared memory with coalesced loads once and read
// by every right-hand side (one warp per right-hand side, conflict-free [entry][tet] layout).
constexpr int kCacheTets = 32;

__global__ void __launch_bounds__(kCacheTets* kCutMaxR)
    k_apply_cut_cached(const float* __restrict__ d, float* __restrict__ q, const CutData cd,
                       const float* __restrict__ kc, const ApplyArgs a, int r0, int nr) {
  __shared__ float sK[kCutPacked * kCacheTets];
  __shared__ double acc[kCutMaxR];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + kCacheTets * ty, nth = kCacheTets * nr;
  const int rhs = r0 + ty;
  const bool act = !a.active || a.active[rhs];
  if (a.units_cut && tid == 0 && blockIdx.x == 0) {
    unsigned long long n = 0;
    for (int rr = 0; rr < nr; ++rr) n += (!a.active || a.active[r0 + rr]) ? 1 : 0;
    atomicAdd(a.units_cut, n);
  }
  const long long N = a.g.N;
  const int nX = a.nX, ncut = cd.ncut;
  const float* dr = d + rhs * a.stride;
  float* qr = q + rhs * a.stride;
  float en = 0.0f;
  for (int base = blockIdx.x * kCacheTets; base < ncut; base += gridDim.x * kCacheTets) {
    __syncthreads();  // the previous group's matrices are no longer read
    for (int i = tid; i < kCutPacked * kCacheTets; i += nth) {
      const int k = i / kCacheTets, tt = i - k * kCacheTets;
      const int e = base + tt;
      sK[i] = e < ncut ? kc[(long long)k * ncut + e] : 0.0f;
    }
    __syncthreads();
    const int e = base + tx;
    if (e < ncut && act) {
      int nd[4], ei[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        nd[k] = cd.ip[k * ncut + e];
        ei[k] = cd.ip[(4 + k) * ncut + e];
      }
      float de[24], qe[24];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          de[3 * k + c] = dr[c * N + nd[k]];
          de[12 + 3 * k + c] = dr[3 * N + (long long)c * nX + ei[k]];
        }
#pragma unroll
      for (int i = 0; i < 24; ++i) qe[i] = 0.0f;
      const float* Kt = sK + tx;
#pragma unroll
      for (int i = 0; i < 24; ++i) {
#pragma unroll
        for (int j = i; j < 24; ++j) {
          const float kij = Kt[(i * 24 - (i * (i - 1)) / 2 + (j - i)) * kCacheTets];
          qe[i] += kij * de[j];
          if (j != i) qe[j] += kij * de[i];
        }
      }
#pragma unroll
      for (int i = 0; i < 24; ++i) en += de[i] * qe[i];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          atomicAdd(&qr[c * N + nd[k]], qe[3 * k + c]);
          atomicAdd(&qr[3 * N + (long long)c * nX + ei[k]], qe[12 + 3 * k + c]);
        }
    }
  }
  // <d, q> per right-hand side: one warp per right-hand side (every acc[ty < nr] is written)
  const double w = (double)warp_sum(en);
  if (tx == 0) acc[ty] = w;
  __syncthreads();
  for (int i = tid; i < nr * 7; i += nth) {
    const int rr = i / 7, k = i - rr * 7;
    if (a.active && !a.active[r0 + rr]) continue;
    a.partials[((long long)(r0 + rr) * 7 + k) * a.nparts + a.part_offset_cut + blockIdx.x] =
        k == 0 ? acc[rr] : 0.0;
  }
}

static cudaError_t launch_cut_cached(const float* d, float* q, CutData cd, const ApplyArgs& a, int n_rhs,
                                     cudaStream_t s) {
  const int nb = apply_cut_blocks(cd.ncut);
  for (int r0 = 0; r0 < n_rhs; r0 += kCutMaxR) {
    const int nr = n_rhs - r0 < kCutMaxR ? n_rhs - r0 : kCutMaxR;
    k_apply_cut_cached<<<nb, dim3(kCacheTets, nr), 0, s>>>(d, q, cd, a.kcache, a, r0, nr);
  }
  return cudaGetLastError();
}

// The enriched part of q only receives atomic contributions from the cut-tet kernel: it is
// cleared first; the standard part must already hold the uncut kernel's plain stores.
template <typename T>
cudaError_t launch_apply_cut(const typename Store<T>::type* d, typename Store<T>::type* q,
                             const typename Store<T>::type* isD, CutData cd, const ApplyArgs& a,
                             int n_rhs, cudaStream_t s) {
  typedef typename Store<T>::type S;
  const GridDev& g = a.g;
  if (a.nX > 0) {
    for (int r = 0; r < n_rhs; ++r) {
      cudaError_t e = cudaMemsetAsync(q + r * a.stride + 3 * g.N, 0, sizeof(S) * 3 * (size_t)a.nX, s);
      if (e != cudaSuccess) return e;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if (a.kcache && !a.eps && !a.want_sig && cd.ncut > 0) return launch_cut_cached(d, q, cd, a, n_rhs, s);
  }
  // launched even without cut tets: its blocks write the (zero) partial sums of their slots
  const int nb = a.cut_blocks > 0 ? a.cut_blocks : apply_cut_blocks(cd.ncut);
  const int rpl = a.cut_rpl > 0 && a.cut_rpl < kCutMaxR ? a.cut_rpl : kCutMaxR;
  const bool sig = a.want_sig || a.eps;
  constexpr size_t smem = cut_smem_bytes<T>();
  // opt in to the staged records' shared memory, once per variant and device
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return ed;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_apply_cut<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_apply_cut<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_apply_cut<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  for (int r0 = 0; r0 < n_rhs; r0 += rpl) {
    const int nr = n_rhs - r0 < rpl ? n_rhs - r0 : rpl;
    if (a.eps)
      k_apply_cut<T, true, true><<<nb, kCutThreads, smem, s>>>(d, q, cd, a, r0, nr);
    else if (sig)
      k_apply_cut<T, false, true><<<nb, kCutThreads, smem, s>>>(d, q, cd, a, r0, nr);
    else
      k_apply_cut<T, false, false><<<nb, kCutThreads, smem, s>>>(d, q, cd, a, r0, nr);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const typename Store<T>::type* d, typename Store<T>::type* q,
                         const typename Store<T>::type* isD, CutData cd, const ApplyArgs& a,
                         int n_rhs, cudaStream_t s) {
  cudaError_t e = launch_apply_uncut<T>(d, q, a, n_rhs, s);
  if (e != cudaSuccess) return e;
  return launch_apply_cut<T>(d, q, isD, cd, a, n_rhs, s);
}

#define XFFT_INST(T)                                                                             \
  template cudaError_t launch_apply<T>(const Store<T>::type*, Store<T>::type*,                  \
                                       const Store<T>::type*, CutData, const ApplyArgs&, int,   \
                                       cudaStream_t);                                           \
  template cudaError_t launch_apply_uncut<T>(const Store<T>::type*, Store<T>::type*,            \
                                             const ApplyArgs&, int, cudaStream_t);              \
  template cudaError_t launch_apply_cut<T>(const Store<T>::type*, Store<T>::type*,              \
                                           const Store<T>::type*, CutData, const ApplyArgs&, int, \
                                           cudaStream_t);
XFFT_INST(float)
XFFT_INST(double)
XFFT_INST(dw)
#undef XFFT_INST
XFFT_APPLY_INST_NPH(, float, 2)
XFFT_APPLY_INST_NPH(, double, 2)
XFFT_APPLY_INST_NPH(, dw, 2)

// ---------------------------------------------------------------- per-voxel average stress
__global__ void k_voxel_stress_uncut(const double* __restrict__ u, const ApplyArgs a,
                                     double* __restrict__ out) {
  const int rhs = blockIdx.y;
  const GridDev& g = a.g;
  const double* ur = u + rhs * a.stride;
  double E[6];
  mandel_to_tensor(a.eps + 6 * rhs, E);
  double ih[3], w[3];
  for (int k = 0; k < 3; ++k) {
    ih[k] = 1.0 / g.h[k];
    w[k] = g.vol_tet / g.h[k];
  }
  const double ivox = 1.0 / (6.0 * g.vol_tet);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.N;
       v += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(v % g.n2);
    const int j = (int)((v / g.n2) % g.n1);
    const int i = (int)(v / ((long long)g.n1 * g.n2));
    double uu[8][3];
    for (int c = 0; c < 8; ++c) {
      const long long nd = corner_node(g, i, j, k, c);
      for (int x = 0; x < 3; ++x) uu[c][x] = ur[x * g.N + nd];
    }
    const double sv = a.scale ? (double)a.scale[v] : 1.0;
    double lms[kMaxPhases], mus[kMaxPhases];
    for (int p = 0; p < kMaxPhases; ++p) {
      lms[p] = a.ph.lam[p] * sv;
      mus[p] = a.ph.mu[p] * sv;
    }
    double F[8][3] = {};
    double en = 0.0, sg[6] = {0, 0, 0, 0, 0, 0};
    const unsigned code = a.code[v];
    tet_uncut<double, 0, true>(uu, F, code, lms, mus, ih, w, g.vol_tet, E, en, sg);
    tet_uncut<double, 1, true>(uu, F, code, lms, mus, ih, w, g.vol_tet, E, en, sg);
    tet_uncut<double, 2, true>(uu, F, code, lms, mus, ih, w, g.vol_tet, E, en, sg);
    tet_uncut<double, 3, true>(uu, F, code, lms, mus, ih, w, g.vol_tet, E, en, sg);
    tet_uncut<double, 4, true>(uu, F, code, lms, mus, ih, w, g.vol_tet, E, en, sg);
    tet_uncut<double, 5, true>(uu, F, code, lms, mus, ih, w, g.vol_tet, E, en, sg);
    const double r2 = 1.41421356237309504880;
    double* o = out + (long long)rhs * 6 * g.N;
    o[0 * g.N + v] = sg[0] * ivox;
    o[1 * g.N + v] = sg[1] * ivox;
    o[2 * g.N + v] = sg[2] * ivox;
    o[3 * g.N + v] = sg[3] * r2 * ivox;
    o[4 * g.N + v] = sg[4] * r2 * ivox;
    o[5 * g.N + v] = sg[5] * r2 * ivox;
  }
}

__global__ void k_voxel_stress_cut(const double* __restrict__ u, const double* __restrict__ isD,
                                   const CutData cd, const ApplyArgs a, double* __restrict__ out) {
  const int rhs = blockIdx.y;
  const GridDev& g = a.g;
  const long long N = g.N;
  const int nX = a.nX, ncut = cd.ncut;
  const double* ur = u + rhs * a.stride;
  double E[6];
  mandel_to_tensor(a.eps + 6 * rhs, E);
  double ih[3];
  for (int k = 0; k < 3; ++k) ih[k] = 1.0 / g.h[k];
  const double ivox = 1.0 / (6.0 * g.vol_tet);
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
    double us[4][3], ws[4][3];
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) {
        us[k][c] = ur[c * N + nd[k]];
        ws[k][c] = ur[3 * N + (long long)c * nX + ei[k]] * isD[(long long)c * nX + ei[k]];
      }
    double L[4];
    for (int b = 0; b < 4; ++b) L[b] = cd.dp[(long long)cut_f_L(b) * ncut + e];
    const double sv = a.scale ? (double)a.scale[vox] : 1.0;
    double es[6] = {0, 0, 0, 0, 0, 0}, ew[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) {
      es[0] += us[k][0] * gr[k][0];
      es[1] += us[k][1] * gr[k][1];
      es[2] += us[k][2] * gr[k][2];
      es[3] += 0.5 * (us[k][1] * gr[k][2] + us[k][2] * gr[k][1]);
      es[4] += 0.5 * (us[k][0] * gr[k][2] + us[k][2] * gr[k][0]);
      es[5] += 0.5 * (us[k][0] * gr[k][1] + us[k][1] * gr[k][0]);
      ew[0] += ws[k][0] * gr[k][0];
      ew[1] += ws[k][1] * gr[k][1];
      ew[2] += ws[k][2] * gr[k][2];
      ew[3] += 0.5 * (ws[k][1] * gr[k][2] + ws[k][2] * gr[k][1]);
      ew[4] += 0.5 * (ws[k][0] * gr[k][2] + ws[k][2] * gr[k][0]);
      ew[5] += 0.5 * (ws[k][0] * gr[k][1] + ws[k][1] * gr[k][0]);
    }
    for (int k = 0; k < 6; ++k) es[k] += E[k];
    double tot[6] = {0, 0, 0, 0, 0, 0};
    for (int si = 0; si < 2; ++si) {
      const double s = si == 0 ? 1.0 : -1.0;
      const int ph = si == 0 ? cut_phase_plus(sph) : cut_phase_minus(sph);
      const double lam = a.ph.lam[ph] * sv, mu = a.ph.mu[ph] * sv;
      double c[4], gam[3] = {0, 0, 0};
      for (int b = 0; b < 4; ++b) {
        c[b] = fabs(L[b]) - s * L[b];
        for (int x = 0; x < 3; ++x) gam[x] += c[b] * gr[b][x];
      }
      for (int b = 0; b < 4; ++b) {
        const double mb = cd.dp[(long long)cut_f_m(si, b) * ncut + e];
        const double* wb = ws[b];
        double eb[6] = {es[0] + c[b] * ew[0] + wb[0] * gam[0], es[1] + c[b] * ew[1] + wb[1] * gam[1],
                        es[2] + c[b] * ew[2] + wb[2] * gam[2],
                        es[3] + c[b] * ew[3] + 0.5 * (wb[1] * gam[2] + wb[2] * gam[1]),
                        es[4] + c[b] * ew[4] + 0.5 * (wb[0] * gam[2] + wb[2] * gam[0]),
                        es[5] + c[b] * ew[5] + 0.5 * (wb[0] * gam[1] + wb[1] * gam[0])};
        double sb[6];
        iso_stress(eb, lam, mu, sb);
        for (int k = 0; k < 6; ++k) tot[k] += mb * sb[k];
      }
    }
    const double r2 = 1.41421356237309504880;
    double* o = out + (long long)rhs * 6 * N;
    atomicAdd(&o[0 * N + vox], tot[0] * ivox);
    atomicAdd(&o[1 * N + vox], tot[1] * ivox);
    atomicAdd(&o[2 * N + vox], tot[2] * ivox);
    atomicAdd(&o[3 * N + vox], tot[3] * r2 * ivox);
    atomicAdd(&o[4 * N + vox], tot[4] * r2 * ivox);
    atomicAdd(&o[5 * N + vox], tot[5] * r2 * ivox);
  }
}

cudaError_t launch_voxel_stress(const double* u, const double* isD, CutData cd,
                                const ApplyArgs& a, double* out, int n_rhs, cudaStream_t s) {
  long long nb = (a.g.N + 255) / 256;
  if (nb > 65535) nb = 65535;
  k_voxel_stress_uncut<<<dim3((unsigned)nb, n_rhs), 256, 0, s>>>(u, a, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || cd.ncut == 0) return e;
  k_voxel_stress_cut<<<dim3(apply_cut_blocks(cd.ncut), n_rhs), 128, 0, s>>>(u, isD, cd, a, out);
  return cudaGetLastError();
}

}  // namespace xfft
