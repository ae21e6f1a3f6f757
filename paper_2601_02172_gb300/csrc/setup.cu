// Setup kernels of the X-FFT solver: snapping, cut-tet classification, enriched-node
// numbering, per-side sub-tetrahedron moments and the scaling factors D0.
//
//  * Snap (Sec. 3): |L_i| < tau counts as on the interface, L_i <- 0.
//  * A P1 tet is cut iff its nodal level-set values take both signs (the modified abs
//    enrichment, eq. modifiedabsEnrichment, vanishes identically otherwise); the enriched
//    nodes J are all nodes of cut tets (eq. X-FEM_space).  Enriched ids follow the node order.
//  * Several interfaces (K level sets, Sec. 4.2's coated sphere): a point lies in phase k if
//    L_k is the first negative level set there, in phase K if none is.  A tet's first level set
//    that is negative at a vertex gives the phase of an uncut tet; if that level set also takes
//    a positive value the tet is cut by its interface, the minus side in phase k and the plus
//    side in the first later level set negative on the tet (else K).  One interface per
//    element: a later level set changing sign on a cut tet is an error.  Each cut tet is
//    enriched with the modified abs of its own interface's level set.
//  * Each side s of a cut tet (s = +: L_h > 0, s = -: L_h < 0) is a tetrahedron or a
//    triangular prism bounded by the linearised interface L_h = 0 (Sec. 3, Fig. subdivision).
//    Instead of quadrature points we store its exact moments int N_b and int N_b N_c of the
//    parent P1 functions; every integrand of the method is a quadratic in the N_b on a side,
//    so these moments reproduce the paper's exact sub-tetrahedron quadrature.
//  * D0 per enriched DOF (node j, component k): int |sym(grad N_X^j (x) e_k)|^2
//    (eq. XFFT_diagonal with the symmetrised gradient of the vector shape function).
#include <cuda_runtime.h>
#include <stdint.h>

#include "cut_geometry.cuh"
#include "xfft_kernels.h"

namespace xfft {

// ---------------------------------------------------------------- snap + classify
__global__ void k_snap(const double* __restrict__ L, double* __restrict__ Ls, long long N,
                       double tau) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = L[i];
    Ls[i] = fabs(v) < tau ? 0.0 : v;
  }
}

__global__ void k_classify(const double* __restrict__ Ls, int nL, GridDev g, uint16_t* __restrict__ code,
                           int* __restrict__ cutcount, int* __restrict__ enr_flag, int* __restrict__ bad,
                           int p1) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.N;
       v += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(v % g.n2);
    const int j = (int)((v / g.n2) % g.n1);
    const int i = (int)(v / ((long long)g.n1 * g.n2));
    double Lc[kMaxPhases - 1][8];
    long long nd[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) nd[c] = corner_node(g, i, j, k, c);
    for (int l = 0; l < nL; ++l)
#pragma unroll
      for (int c = 0; c < 8; ++c) Lc[l][c] = Ls[l * g.N + nd[c]];
    if (p1) {
      // P1 baseline (voxel-segmented, no enrichment): the voxel takes the phase of its centre,
      // where the trilinear interpolant of the corner values is their mean; the first level
      // set negative there decides (phase nL if none is)
      int ph = nL;
      for (int l = nL - 1; l >= 0; --l) {
        double m = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) m += Lc[l][c];
        if (m * 0.125 < 0.0) ph = l;
      }
      const unsigned pc = phase_code(ph);
      unsigned cd = 0;
#pragma unroll
      for (int t = 0; t < 6; ++t) cd |= pc << (2 * t);
      code[v] = (uint16_t)cd;
      cutcount[v] = 0;
      continue;
    }
    unsigned cd = 0;
    int cnt = 0;
    bool two = false;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      double tv[kMaxPhases - 1][4];
      const double* pv[kMaxPhases - 1];
      for (int l = 0; l < nL; ++l) {
        tv[l][0] = Lc[l][0];
        tv[l][1] = Lc[l][tet_c1(t)];
        tv[l][2] = Lc[l][tet_c2(t)];
        tv[l][3] = Lc[l][7];
        pv[l] = tv[l];
      }
      int pm, pp;
      const unsigned bits = classify_tet(pv, nL, &pm, &pp, &two);
      if (bits == kCodeCut) {
        ++cnt;
        enr_flag[nd[0]] = 1;
        enr_flag[nd[tet_c1(t)]] = 1;
        enr_flag[nd[tet_c2(t)]] = 1;
        enr_flag[nd[7]] = 1;
      }
      cd |= bits << (2 * t);
    }
    code[v] = (uint16_t)cd;
    cutcount[v] = cnt;
    if (two) atomicAdd(bad, 1);
  }
}

// number of non-finite level-set values and of non-finite scale values (host validation)
__global__ void k_count_nonfinite(const double* __restrict__ L, long long nL, const float* __restrict__ sc,
                                  long long ns, int* __restrict__ out) {
  int bl = 0, bs = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nL;
       i += (long long)gridDim.x * blockDim.x)
    bl += isfinite(L[i]) ? 0 : 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns;
       i += (long long)gridDim.x * blockDim.x)
    bs += isfinite(sc[i]) ? 0 : 1;
  if (bl) atomicAdd(out, bl);
  if (bs) atomicAdd(out + 1, bs);
}

cudaError_t launch_count_nonfinite(const double* L, long long nL, const float* sc, long long ns,
                                   int* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  long long nb = ((nL > ns ? nL : ns) + kThreads - 1) / kThreads;
  if (nb > 152 * 16) nb = 152 * 16;
  if (nb < 1) nb = 1;
  k_count_nonfinite<<<(int)nb, kThreads, 0, s>>>(L, nL, sc, sc ? ns : 0, out);
  return cudaGetLastError();
}

cudaError_t launch_snap_classify(const double* L, double* Ls, int nL, uint16_t* code, int* cutcount,
                                 int* enr_flag, int* bad, GridDev g, double tau, int p1, cudaStream_t s) {
  if (nL < 1 || nL > kMaxPhases - 1) return cudaErrorInvalidValue;
  const int nb = (int)((g.N + kThreads - 1) / kThreads);
  const int grid = nb < 65535 * 16 ? nb : 65535 * 16;
  cudaError_t e = cudaMemsetAsync(enr_flag, 0, sizeof(int) * g.N, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_snap<<<grid, kThreads, 0, s>>>(L, Ls, nL * g.N, tau);
  k_classify<<<grid, kThreads, 0, s>>>(Ls, nL, g, code, cutcount, enr_flag, bad, p1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- exclusive scan (int32)
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ inline int block_exclusive_scan(int v, int* smem, int* total) {
  // returns the exclusive prefix of v over the block; *total receives the block sum
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? smem[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) smem[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const int before = wid > 0 ? smem[wid - 1] : 0;
  *total = smem[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

// Phase 1/3: each block scans one tile in place (exclusive) and records its total.
// in and out may alias (in-place scan): no __restrict__ on them
__global__ void k_scan_tiles(const int* in, int* out, long long n, int* __restrict__ tile_sums) {
  __shared__ int smem[32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int vals[kScanItems];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long idx = base + k;
    vals[k] = idx < n ? in[idx] : 0;
    sum += vals[k];
  }
  int total;
  int run = block_exclusive_scan(sum, smem, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long idx = base + k;
    if (idx < n) out[idx] = run;
    run += vals[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Phase 2: one block scans the tile sums (exclusive) and writes the grand total.
__global__ void k_scan_sums(int* __restrict__ sums, int nt, int* __restrict__ total_out) {
  __shared__ int smem[32];
  const int per = (nt + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  int local = 0;
  for (int k = 0; k < per; ++k)
    if (beg + k < nt) local += sums[beg + k];
  int total;
  int run = block_exclusive_scan(local, smem, &total);
  for (int k = 0; k < per; ++k) {
    if (beg + k < nt) {
      const int v = sums[beg + k];
      sums[beg + k] = run;
      run += v;
    }
  }
  if (threadIdx.x == 0) *total_out = total;
}

__global__ void k_scan_add(int* __restrict__ out, long long n, const int* __restrict__ sums) {
  const int add = sums[blockIdx.x];
  const long long base = (long long)blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    const long long idx = base + k;
    if (idx < n) out[idx] += add;
  }
}

size_t scan_tmp_ints(long long n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 32; }

cudaError_t launch_scan(const int* in, int* out, long long n, int* d_total, int* d_tmp,
                        cudaStream_t s) {
  const long long nt = (n + kScanTile - 1) / kScanTile;
  if (nt > (1LL << 30)) return cudaErrorInvalidValue;
  k_scan_tiles<<<(unsigned)nt, kThreads, 0, s>>>(in, out, n, d_tmp);
  k_scan_sums<<<1, 1024, 0, s>>>(d_tmp, (int)nt, d_total);
  k_scan_add<<<(unsigned)nt, kThreads, 0, s>>>(out, n, d_tmp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- lists
__global__ void k_enr_lists(const int* __restrict__ enr_flag, int* __restrict__ enr_id,
                            int* __restrict__ enr_nodes, GridDev g) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.N;
       v += (long long)gridDim.x * blockDim.x) {
    // enr_id holds the exclusive scan of enr_flag on entry
    if (enr_flag[v]) {
      enr_nodes[enr_id[v]] = (int)v;
    } else {
      enr_id[v] = -1;
    }
  }
}

// cut flags of Kuhn tet t per voxel (t < 0: the voxel has some cut tet)
__global__ void k_tet_flags(const uint16_t* __restrict__ code, int t, int* __restrict__ flags, long long N) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    const unsigned cd = code[v];
    int f = 0;
    if (t >= 0) {
      f = ((cd >> (2 * t)) & 3u) == kCodeCut;
    } else {
      for (int k = 0; k < 6; ++k) f |= ((cd >> (2 * k)) & 3u) == kCodeCut;
    }
    flags[v] = f;
  }
}

// first voxel of each chunk of kChunkVoxels consecutive cut voxels (rank = exclusive scan of the
// cut-voxel flags); first[nchunks] = N
#ifndef XFFT_CHUNK_VOXELS
#define XFFT_CHUNK_VOXELS 2048
#endif
constexpr int kChunkVoxels = XFFT_CHUNK_VOXELS;
__global__ void k_chunk_first(const uint16_t* __restrict__ code, const int* __restrict__ rank,
                              const int* __restrict__ ncv, int* __restrict__ first, long long N) {
  const int nchunks = (*ncv + kChunkVoxels - 1) / kChunkVoxels;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    const unsigned cd = code[v];
    bool cut = false;
    for (int k = 0; k < 6; ++k) cut |= ((cd >> (2 * k)) & 3u) == kCodeCut;
    if (cut && rank[v] % kChunkVoxels == 0) first[rank[v] / kChunkVoxels] = (int)v;
    if (v == 0) first[nchunks] = (int)N;
  }
}

// acc[k] = position of chunk k's first cut tet (voxel order, cutoff = scan of per-voxel counts)
__global__ void k_chunk_init(const int* __restrict__ first, const int* __restrict__ cutoff,
                             const int* __restrict__ ncv, int* __restrict__ acc) {
  const int nchunks = (*ncv + kChunkVoxels - 1) / kChunkVoxels;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nchunks; k += gridDim.x * blockDim.x)
    acc[k] = cutoff[first[k]];
}

__device__ inline int chunk_of(const int* __restrict__ first, int nchunks, long long v) {
  int lo = 0, hi = nchunks - 1;  // largest k with first[k] <= v
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// cut tets of type t: position acc[chunk] + (their rank among the chunk's voxels cut there);
// P = exclusive scan of the type-t flags
__global__ void k_place_tets(const uint16_t* __restrict__ code, const int* __restrict__ P, int t,
                             const int* __restrict__ first, const int* __restrict__ acc,
                             const int* __restrict__ ncv, int* __restrict__ cut_ints, int ncut, long long N) {
  const int nchunks = (*ncv + kChunkVoxels - 1) / kChunkVoxels;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
       v += (long long)gridDim.x * blockDim.x) {
    if (((code[v] >> (2 * t)) & 3u) != kCodeCut) continue;
    const int k = chunk_of(first, nchunks, v);
    const int e = acc[k] + P[v] - P[first[k]];
    cut_ints[8 * ncut + e] = (int)v;  // voxel
    cut_ints[9 * ncut + e] = t;       // tet
  }
}

// acc[k] += number of type-t cut tets in chunk k
__global__ void k_chunk_advance(const int* __restrict__ P, const int* __restrict__ total_t,
                                const int* __restrict__ first, const int* __restrict__ ncv,
                                int* __restrict__ acc, long long N) {
  const int nchunks = (*ncv + kChunkVoxels - 1) / kChunkVoxels;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nchunks; k += gridDim.x * blockDim.x) {
    const int hi = first[k + 1] >= N ? *total_t : P[first[k + 1]];
    acc[k] += hi - P[first[k]];
  }
}

int chunk_ints(int ncut) { return ncut / kChunkVoxels + 2; }

// Enriched numbering, then the cut-tet list in chunks of kChunkVoxels consecutive cut voxels,
// inside a chunk grouped by Kuhn tet type (voxel order within a type): the apply kernels then run
// one compile-time tet type per warp (except at the few group boundaries) while a chunk's node
// data stays in cache.  work: N ints (enr_flag's storage, free once the enriched ids exist);
// cutoff: exclusive scan of the per-voxel cut-tet counts; tot: 7 device ints; first, acc:
// chunk_ints(ncut) ints each.
cudaError_t launch_build_lists(const uint16_t* code, const int* cutoff, int* enr_flag, int* enr_id,
                               int* enr_nodes, int* cut_ints, int ncut, GridDev g, int* tot,
                               int* scan_tmp, int* first, int* acc, cudaStream_t s) {
  const int nb = (int)((g.N + kThreads - 1) / kThreads);
  const int grid = nb < 65535 * 16 ? nb : 65535 * 16;
  k_enr_lists<<<grid, kThreads, 0, s>>>(enr_flag, enr_id, enr_nodes, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || ncut == 0) return e;
  int* work = enr_flag;
  int* ncv = tot + 6;
  k_tet_flags<<<grid, kThreads, 0, s>>>(code, -1, work, g.N);
  e = launch_scan(work, work, g.N, ncv, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_chunk_first<<<grid, kThreads, 0, s>>>(code, work, ncv, first, g.N);
  const int cb = (chunk_ints(ncut) + kThreads - 1) / kThreads;
  k_chunk_init<<<cb, kThreads, 0, s>>>(first, cutoff, ncv, acc);
  e = cudaGetLastError();
  for (int t = 0; t < 6 && e == cudaSuccess; ++t) {
    k_tet_flags<<<grid, kThreads, 0, s>>>(code, t, work, g.N);
    e = launch_scan(work, work, g.N, tot + t, scan_tmp, s);
    if (e == cudaSuccess) {
      k_place_tets<<<grid, kThreads, 0, s>>>(code, work, t, first, acc, ncv, cut_ints, ncut, g.N);
      k_chunk_advance<<<cb, kThreads, 0, s>>>(work, tot + t, first, ncv, acc, g.N);
      e = cudaGetLastError();
    }
  }
  return e;
}

__global__ void k_cut_geometry(const double* __restrict__ Ls, int nL, int* __restrict__ ip,
                               double* __restrict__ dp, int ncut, GridDev g) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncut; e += gridDim.x * blockDim.x) {
    const long long v = ip[8 * ncut + e];
    const int t = ip[9 * ncut + e];
    const int k = (int)(v % g.n2);
    const int j = (int)((v / g.n2) % g.n1);
    const int i = (int)(v / ((long long)g.n1 * g.n2));
    long long nd[4];
    double tv[kMaxPhases - 1][4];
    const double* pv[kMaxPhases - 1];
    for (int a = 0; a < 4; ++a) {
      nd[a] = corner_node(g, i, j, k, tet_corner(t, a));
      ip[a * ncut + e] = (int)nd[a];
    }
    for (int l = 0; l < nL; ++l) {
      for (int a = 0; a < 4; ++a) tv[l][a] = Ls[l * g.N + nd[a]];
      pv[l] = tv[l];
    }
    // the cutting interface is the tet's first level set with a negative vertex
    int pm = 0, pp = 1;
    bool two = false;
    classify_tet(pv, nL, &pm, &pp, &two);
    ip[kCutFieldPhases * ncut + e] = pm | (pp << 8);
    double L[4];
    for (int a = 0; a < 4; ++a) {
      L[a] = tv[pm][a];
      dp[cut_f_L(a) * (long long)ncut + e] = L[a];
    }
    for (int si = 0; si < 2; ++si) {
      Moments mo;
      side_moments(L, si == 0 ? +1 : -1, g.vol_tet, mo);
      for (int b = 0; b < 4; ++b) dp[cut_f_m(si, b) * (long long)ncut + e] = mo.m[b];
      for (int c = 0; c < 10; ++c) dp[cut_f_M(si, c) * (long long)ncut + e] = mo.M[c];
    }
  }
}

__global__ void k_cut_eids(int* __restrict__ ip, const int* __restrict__ enr_id, int ncut) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncut; e += gridDim.x * blockDim.x) {
    for (int a = 0; a < 4; ++a) ip[(4 + a) * ncut + e] = enr_id[ip[a * ncut + e]];
  }
}

cudaError_t launch_cut_geometry(const double* Ls, int nL, CutData cd, double* dp_mut, int* ip_mut,
                                GridDev g, cudaStream_t s) {
  if (cd.ncut == 0) return cudaSuccess;
  const int nb = (cd.ncut + 127) / 128;
  k_cut_geometry<<<nb, 128, 0, s>>>(Ls, nL, ip_mut, dp_mut, cd.ncut, g);
  return cudaGetLastError();
}

// enr ids of the cut-tet nodes (needs enr_id); called after launch_cut_geometry
cudaError_t launch_cut_eids(int* ip_mut, const int* enr_id, int ncut, cudaStream_t s) {
  if (ncut == 0) return cudaSuccess;
  k_cut_eids<<<(ncut + 255) / 256, 256, 0, s>>>(ip_mut, enr_id, ncut);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- scaling factors D0
// On side s of a cut tet, grad N_X^a(x) = sum_b N_b(x) V_ab with V_ab = c_b g_a + delta_ab gamma,
// c_b = |L_b| - s L_b, gamma = sum_b c_b g_b.  Hence
//   D_{a,k} += 1/2 sum_bc M_bc (V_ab . V_ac + V_ab[k] V_ac[k]).
// D (3 x nX): D0 per enriched DOF; Doff (3 x nX, may be null): the off-diagonal entries
// (01, 02, 12) of each enriched node's 3x3 block int sym(g (x) e_k) : sym(g (x) e_l) = 1/2 int
// g_k g_l (k != l), g = grad N_X (used by the block enriched preconditioner)
__global__ void k_cut_scaling(const int* __restrict__ ip, const double* __restrict__ dp, int ncut,
                              double* __restrict__ D, double* __restrict__ Doff, int nX, GridDev g) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncut; e += gridDim.x * blockDim.x) {
    const int t = ip[9 * ncut + e];
    double ih[3] = {1.0 / g.h[0], 1.0 / g.h[1], 1.0 / g.h[2]};
    double gr[4][3];
    tet_grads<double>(t, ih, gr);
    double L[4], Mp[2][10];
    for (int b = 0; b < 4; ++b) L[b] = dp[cut_f_L(b) * (long long)ncut + e];
    for (int si = 0; si < 2; ++si)
      for (int k = 0; k < 10; ++k) Mp[si][k] = dp[cut_f_M(si, k) * (long long)ncut + e];
    double acc[4][3], off[4][3];
    cut_scaling_terms(L, gr, Mp, acc, off, Doff != nullptr);
    for (int a = 0; a < 4; ++a) {
      const int j = ip[(4 + a) * ncut + e];
      for (int x = 0; x < 3; ++x) atomicAdd(&D[(long long)x * nX + j], acc[a][x]);
      if (Doff)
        for (int x = 0; x < 3; ++x) atomicAdd(&Doff[(long long)x * nX + j], off[a][x]);
    }
  }
}

__global__ void k_cut_matrix(const int* __restrict__ ip, const double* __restrict__ dp,
                             const double* __restrict__ isD, int nX, int ncut, GridDev g, PhaseDev ph,
                             const float* __restrict__ scale, float* __restrict__ kc) {
  double ih[3];
  for (int k = 0; k < 3; ++k) ih[k] = 1.0 / g.h[k];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncut; e += gridDim.x * blockDim.x) {
    const int vox = ip[8 * ncut + e];
    const int t = ip[9 * ncut + e];
    const int sph = ip[kCutFieldPhases * ncut + e];
    double gr[4][3];
    tet_grads<double>(t, ih, gr);
    double L[4], dsc[4][3];
    for (int a = 0; a < 4; ++a) {
      L[a] = dp[(long long)cut_f_L(a) * ncut + e];
      const int j = ip[(4 + a) * ncut + e];
      for (int x = 0; x < 3; ++x) dsc[a][x] = isD[(long long)x * nX + j];
    }
    const double sv = scale ? (double)scale[vox] : 1.0;
    SideW w[2];
    for (int si = 0; si < 2; ++si) {
      const int p = si == 0 ? cut_phase_plus(sph) : cut_phase_minus(sph);
      double Mp[10];
      for (int k = 0; k < 10; ++k) Mp[k] = dp[(long long)cut_f_M(si, k) * ncut + e];
      side_weights(L, si == 0 ? 1.0 : -1.0, gr, Mp, ph.lam[p] * sv, ph.mu[p] * sv, w[si]);
    }
    int k = 0;
    for (int i = 0; i < 24; ++i)
      for (int j = i; j < 24; ++j, ++k) kc[(long long)k * ncut + e] = (float)cut_element_entry(i, j, w, gr, dsc);
  }
}

__global__ void k_cut_records(const int* __restrict__ ip, const double* __restrict__ dp,
                              const double* __restrict__ isD, int nX, int ncut, GridDev g, PhaseDev ph,
                              const float* __restrict__ scale, int4* __restrict__ n4,
                              int4* __restrict__ e4, double* __restrict__ r64, float* __restrict__ r32) {
  double ih[3];
  for (int k = 0; k < 3; ++k) ih[k] = 1.0 / g.h[k];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncut; e += gridDim.x * blockDim.x) {
    const int vox = ip[8 * ncut + e];
    const int t = ip[9 * ncut + e];
    const int sph = ip[kCutFieldPhases * ncut + e];
    int nd[4], ej[4];
    for (int a = 0; a < 4; ++a) {
      nd[a] = ip[a * ncut + e];
      ej[a] = ip[(4 + a) * ncut + e];
    }
    n4[e] = make_int4(nd[0], nd[1], nd[2], nd[3]);
    e4[e] = make_int4(ej[0], ej[1], ej[2], ej[3]);
    double gr[4][3];
    tet_grads<double>(t, ih, gr);
    const double sv = scale ? (double)scale[vox] : 1.0;
    double R[kRec];
    for (int k = 0; k < kRec; ++k) R[k] = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int x = 0; x < 3; ++x) R[3 * a + x] = isD[(long long)x * nX + ej[a]];
    double L[4];
    for (int b = 0; b < 4; ++b) L[b] = dp[(long long)cut_f_L(b) * ncut + e];
    for (int si = 0; si < 2; ++si) {
      double* S = R + kRecSide + kRecSideLen * si;
      const double sg = si == 0 ? 1.0 : -1.0;
      double M[10], m[4], c[4];
      for (int k = 0; k < 10; ++k) M[k] = dp[(long long)cut_f_M(si, k) * ncut + e];
      for (int b = 0; b < 4; ++b) {
        m[b] = dp[(long long)cut_f_m(si, b) * ncut + e];
        c[b] = fabs(L[b]) - sg * L[b];
      }
      double V = 0.0, mc = 0.0, cMc = 0.0, gam[3] = {0.0, 0.0, 0.0};
      for (int b = 0; b < 4; ++b) {
        double P = 0.0;
        for (int cc = 0; cc < 4; ++cc) P += M[midx(b, cc)] * c[cc];
        S[14 + b] = P;
        S[10 + b] = m[b];
        V += m[b];
        mc += m[b] * c[b];
        cMc += P * c[b];
        for (int x = 0; x < 3; ++x) gam[x] += c[b] * gr[b][x];
      }
      for (int k = 0; k < 10; ++k) S[k] = M[k];
      for (int x = 0; x < 3; ++x) S[18 + x] = gam[x];
      const int p = si == 0 ? cut_phase_plus(sph) : cut_phase_minus(sph);
      S[21] = ph.lam[p] * sv;
      S[22] = ph.mu[p] * sv;
      S[23] = V;
      S[24] = mc;
      S[25] = cMc;
    }
    for (int k = 0; k < kRec; ++k) {
      r64[(long long)e * kRec + k] = R[k];
      r32[(long long)e * kRec + k] = (float)R[k];
    }
  }
}

cudaError_t launch_cut_records(CutData cd, const double* isD, int nX, GridDev g, PhaseDev ph,
                               const float* scale, int4* n4, int4* e4, double* r64, float* r32,
                               cudaStream_t s) {
  if (cd.ncut == 0) return cudaSuccess;
  k_cut_records<<<(cd.ncut + 127) / 128, 128, 0, s>>>(cd.ip, cd.dp, isD, nX, cd.ncut, g, ph, scale, n4,
                                                        e4, r64, r32);
  return cudaGetLastError();
}

cudaError_t launch_cut_matrix(CutData cd, const double* isD, int nX, GridDev g, PhaseDev ph,
                              const float* scale, float* kc, cudaStream_t s) {
  if (cd.ncut == 0) return cudaSuccess;
  k_cut_matrix<<<(cd.ncut + 127) / 128, 128, 0, s>>>(cd.ip, cd.dp, isD, nX, cd.ncut, g, ph, scale, kc);
  return cudaGetLastError();
}

cudaError_t launch_cut_scaling(CutData cd, double* D, double* Doff, int nX, GridDev g, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(D, 0, sizeof(double) * 3 * (size_t)nX, s);
  if (e == cudaSuccess && Doff) e = cudaMemsetAsync(Doff, 0, sizeof(double) * 3 * (size_t)nX, s);
  if (e != cudaSuccess || cd.ncut == 0) return e;
  k_cut_scaling<<<(cd.ncut + 127) / 128, 128, 0, s>>>(cd.ip, cd.dp, cd.ncut, D, Doff, nX, g);
  return cudaGetLastError();
}

// Block enriched preconditioner: per enriched node the scaled block B = S Dblk S (S = D0^-1/2,
// unit diagonal) is factorised B = L L^T in FP64 and its inverse L^-T L^-1 stored as (00, 11,
// 22, 01, 02, 12) x nX in FP64 and FP32.  A non-positive pivot sets *bad.
__global__ void k_block_inverse(const double* __restrict__ D, const double* __restrict__ Doff,
                                const double* __restrict__ isd, double* __restrict__ b64,
                                float* __restrict__ b32, int nX, int* __restrict__ bad) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nX; j += gridDim.x * blockDim.x) {
    const double s0 = isd[j], s1 = isd[nX + j], s2 = isd[2 * (long long)nX + j];
    const double a00 = D[j] * s0 * s0, a11 = D[nX + j] * s1 * s1, a22 = D[2 * (long long)nX + j] * s2 * s2;
    const double a10 = Doff[j] * s0 * s1, a20 = Doff[nX + j] * s0 * s2, a21 = Doff[2 * (long long)nX + j] * s1 * s2;
    double v[6];
    const bool ok = block_inverse3(a00, a11, a22, a10, a20, a21, v);
    if (!ok) atomicExch(bad, 1);
    for (int k = 0; k < 6; ++k) {
      b64[(long long)k * nX + j] = v[k];
      b32[(long long)k * nX + j] = (float)v[k];
    }
  }
}

cudaError_t launch_block_inverse(const double* D, const double* Doff, const double* isd, double* b64,
                                 float* b32, int nX, int* bad, cudaStream_t s) {
  if (nX == 0) return cudaSuccess;
  k_block_inverse<<<(nX + 255) / 256, 256, 0, s>>>(D, Doff, isd, b64, b32, nX, bad);
  return cudaGetLastError();
}

__global__ void k_finish_scaling(const double* __restrict__ D, double* __restrict__ isd,
                                 float* __restrict__ isf, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = D[i] > 0.0 ? 1.0 / sqrt(D[i]) : 0.0;
    isd[i] = v;
    isf[i] = (float)v;
  }
}

cudaError_t launch_finish_scaling(const double* D, double* isd, float* isf, int nX,
                                  cudaStream_t s) {
  if (nX == 0) return cudaSuccess;
  const long long n = 3LL * nX;
  k_finish_scaling<<<(int)((n + 255) / 256), 256, 0, s>>>(D, isd, isf, n);
  return cudaGetLastError();
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

cudaError_t launch_cut_to_float(const double* dp, float* fp, long long count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  long long nb = (count + 255) / 256;
  if (nb > 65535LL * 16) nb = 65535LL * 16;
  k_to_float<<<(int)nb, 256, 0, s>>>(dp, fp, count);
  return cudaGetLastError();
}

}  // namespace xfft
