// Shared device-side definitions of the X-FFT GB300 kernels.
//
// Grid and numbering (Sec. 3): n0 x n1 x n2 voxels, periodic nodes node = (i*n1 + j)*n2 + k,
// voxel v has its lowest corner at node v.  Each voxel is split into six P1 tetrahedra
// (Fig. P16): tet t = 0..5 belongs to the permutation (p,q,r) of the axes listed in
// kPerm[t] (lexicographic order) and has the corners 0, e_p, e_p+e_q, (1,1,1).  Voxel corners
// are encoded as c = dx + 2 dy + 4 dz.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace xfft {

constexpr int kThreads = 256;

struct GridDev {
  int n0, n1, n2;
  long long N;       // nodes = voxels
  double h[3];       // voxel edge lengths
  double vol_tet;    // h0 h1 h2 / 6
  double volY;       // cell volume
};

// Phase data passed by value to the kernels.  One level set: phase 0 = minus (L < 0),
// 1 = plus.  K level sets (several interfaces, Sec. 4.2's coated sphere): phase k where L_k is
// the first negative level set, phase K where none is; nph = K + 1 <= kMaxPhases.
constexpr int kMaxPhases = 3;
struct PhaseDev {
  double lam[kMaxPhases];
  double mu[kMaxPhases];
  int nph;
};

// Per-voxel tet codes, 2 bits per Kuhn tet t at bits 2t: 0, 1 and 3 = uncut in phase 0, 1 and
// 2; 2 = cut (handled by the cut-tet kernels).
constexpr unsigned kCodeCut = 2u;
__host__ __device__ constexpr int code_phase(unsigned cd) { return cd == 3u ? 2 : (int)cd; }
__host__ __device__ constexpr unsigned phase_code(int p) { return p == 2 ? 3u : (unsigned)p; }

__host__ __device__ constexpr int perm_p(int t) { return t < 2 ? 0 : (t < 4 ? 1 : 2); }
__host__ __device__ constexpr int perm_q(int t) {
  return t == 0 ? 1 : t == 1 ? 2 : t == 2 ? 0 : t == 3 ? 2 : t == 4 ? 0 : 1;
}
__host__ __device__ constexpr int perm_r(int t) { return 3 - perm_p(t) - perm_q(t); }
// corner codes of the four vertices of tet t
__host__ __device__ constexpr int tet_c1(int t) { return 1 << perm_p(t); }
__host__ __device__ constexpr int tet_c2(int t) { return (1 << perm_p(t)) | (1 << perm_q(t)); }
__host__ __device__ constexpr int tet_corner(int t, int a) {
  return a == 0 ? 0 : a == 1 ? tet_c1(t) : a == 2 ? tet_c2(t) : 7;
}

__host__ __device__ inline int wrapi(int i, int n) {
  // valid for i in [-n, 2n)
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

__host__ __device__ inline long long node_index(int i, int j, int k, int n1, int n2) {
  return ((long long)i * n1 + j) * n2 + k;
}

// node of corner c of voxel (i,j,k), periodic
__host__ __device__ inline long long corner_node(const GridDev& g, int i, int j, int k, int c) {
  return node_index(wrapi(i + (c & 1), g.n0), wrapi(j + ((c >> 1) & 1), g.n1),
                    wrapi(k + ((c >> 2) & 1), g.n2), g.n1, g.n2);
}

// Gradients of the P1 vertex functions of tet t: g0 = -e_p/h_p, g1 = e_p/h_p - e_q/h_q,
// g2 = e_q/h_q - e_r/h_r, g3 = e_r/h_r.
template <typename T>
__host__ __device__ inline void tet_grads(int t, const T ih[3], T g[4][3]) {
  const int p = perm_p(t), q = perm_q(t), r = perm_r(t);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) g[a][c] = T(0);
  g[0][p] = -ih[p];
  g[1][p] = ih[p];
  g[1][q] = -ih[q];
  g[2][q] = ih[q];
  g[2][r] = -ih[r];
  g[3][r] = ih[r];
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV values over the block (any 1D/2D/3D shape, a multiple of 32 threads); thread 0
// receives the totals in out[].  smem must hold NV * 32 doubles.  All threads must call it.
template <int NV>
__device__ inline void block_sum(const double (&v)[NV], double* smem, double (&out)[NV]) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
  const int lane = tid & 31, wid = tid >> 5;
  double w[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) w[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) smem[i * 32 + wid] = w[i];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? smem[i * 32 + lane] : 0.0;
      out[i] = warp_sum(s);
    }
  }
  __syncthreads();
}

// Per-RHS solver state, FP64 scalars (Algorithm 1).
struct RhsState {
  double rr;        // f^T P^-1 f of the current iterate
  double rr0;       // at the start of the (inner) solve
  double dq;        // <A d, d>
  double alpha, beta;
  double sig[6];    // int_Y sigma(u) (Mandel), tracked across iterations
  double sd[6];     // int_Y C grad^s d of the last apply
  double rel;       // inner solves: relative reduction of rr^(1/2) to reach
  int active;       // 1 while iterating
  int iters;        // iterations performed
  int status;       // 0 running/converged, 4 not converged, 5 breakdown
  int converged;
  int dpar;         // which of the two direction buffers holds the last direction d
  double cauchy;    // rr / <d, A d> of the last iteration (Barzilai-Borwein step)
  double rr_prev;   // f^T P^-1 f one iteration earlier (Barzilai-Borwein BB2 step)
  double dd, qq;    // <d, d> and <A d, A d> of the last iteration (Euclidean BB steps)
  double bb_step;   // step in use by the cyclic Barzilai-Borwein rule
};

}  // namespace xfft
