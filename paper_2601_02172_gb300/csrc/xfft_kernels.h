// Host-side prototypes of the kernel launchers (internal to libxfft).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "dw.cuh"
#include "xfft_common.cuh"

namespace xfft {

// Per-cut-tet data, structure of arrays of length ncut.
//   ints   (11 fields): node[a] (a<4), eid[a] (a<4), voxel, tet, side phases (minus phase in
//                       bits 0..7, plus phase in bits 8..15)
//   reals  (32 fields): L[b] (b<4), then for side s = 0 (plus) and 1 (minus):
//                       m[s][b] = int_side N_b (b<4) and M[s][k] = int_side N_b N_c
//                       (k<10, packed (00,01,02,03,11,12,13,22,23,33))
struct CutData {
  const int* ip;
  const double* dp;
  const float* fp;
  int ncut;
  // per cut tet, for the apply kernels: the four node ids and enriched ids (int4 each) and a
  // record of kRec reals (FP32 and FP64 copies; layout below)
  const int4* n4 = nullptr;
  const int4* e4 = nullptr;
  const float* r32 = nullptr;
  const double* r64 = nullptr;
};
// Apply record of a cut tet (tet-major, kRec reals, 16-byte aligned groups):
//   [3a + c]            D0^-1/2 of the enriched DOF (vertex a, component c)
//   kRecSide + 28 s +   side s = 0 (plus, L > 0) or 1 (minus):
//     0..9   M_bc = int_side N_b N_c (packed as midx)
//     10..13 m_b = int_side N_b
//     14..17 P_b = sum_c M_bc c_c with c_c = |L_c| - s L_c (s = +1 plus, -1 minus)
//     18..20 gamma = grad rho on the side = sum_b c_b grad N_b
//     21, 22 lambda, mu of the side's phase times the voxel's modulus scale
//     23..25 V = sum_b m_b, m.c = sum_b m_b c_b (= sum_b P_b), c^T M c; 26, 27 zero
constexpr int kRec = 68;
constexpr int kRecSide = 12;
constexpr int kRecSideLen = 28;
constexpr int kCutInts = 11;
constexpr int kCutFieldPhases = 10;
__host__ __device__ constexpr int cut_phase_minus(int f) { return f & 0xff; }
__host__ __device__ constexpr int cut_phase_plus(int f) { return (f >> 8) & 0xff; }
constexpr int kCutReals = 32;
__host__ __device__ constexpr int cut_f_L(int b) { return b; }
__host__ __device__ constexpr int cut_f_m(int s, int b) { return 4 + 14 * s + b; }
__host__ __device__ constexpr int cut_f_M(int s, int k) { return 8 + 14 * s + k; }
__host__ __device__ constexpr int midx(int b, int c) {
  // packed index of the symmetric 4x4 entry (b,c)
  return b <= c ? (b == 0 ? c : b == 1 ? 3 + c : b == 2 ? 5 + c : 9)
                : (c == 0 ? b : c == 1 ? 3 + b : c == 2 ? 5 + b : 9);
}

// ---- setup (setup.cu)
// nL level sets (node order, nL x N); *bad (device int) counts tets cut by two interfaces
// p1 = 1: the P1 baseline (no cut tets, each voxel in the phase of its centre)
cudaError_t launch_snap_classify(const double* L, double* Ls, int nL, uint16_t* code, int* cutcount,
                                 int* enr_flag, int* bad, GridDev g, double tau, int p1, cudaStream_t s);
// out[0] = non-finite values among L (nL doubles), out[1] among sc (ns floats; sc may be null)
cudaError_t launch_count_nonfinite(const double* L, long long nL, const float* sc, long long ns,
                                   int* out, cudaStream_t s);
// exclusive scan of n ints into out (may alias in); writes the total to *d_total (device)
cudaError_t launch_scan(const int* in, int* out, long long n, int* d_total, int* d_tmp,
                        cudaStream_t s);
size_t scan_tmp_ints(long long n);
// enriched ids and nodes, and the cut-tet list (voxel, tet) in chunks of consecutive cut voxels,
// grouped by Kuhn tet type inside a chunk.  enr_flag is used as scratch afterwards; cutoff: the
// exclusive scan of the per-voxel cut-tet counts; tot: 7 device ints; scan_tmp: scan_tmp_ints(N);
// first, acc: chunk_ints(ncut) device ints each
cudaError_t launch_build_lists(const uint16_t* code, const int* cutoff, int* enr_flag, int* enr_id,
                               int* enr_nodes, int* cut_ints, int ncut, GridDev g, int* tot,
                               int* scan_tmp, int* first, int* acc, cudaStream_t s);
int chunk_ints(int ncut);
cudaError_t launch_cut_geometry(const double* Ls, int nL, CutData cd, double* dp_mut, int* ip_mut,
                                GridDev g, cudaStream_t s);
cudaError_t launch_cut_eids(int* ip_mut, const int* enr_id, int ncut, cudaStream_t s);
cudaError_t launch_cut_scaling(CutData cd, double* D, double* Doff, int nX, GridDev g, cudaStream_t s);
cudaError_t launch_block_inverse(const double* D, const double* Doff, const double* isd, double* b64,
                                 float* b32, int nX, int* bad, cudaStream_t s);
cudaError_t launch_finish_scaling(const double* D, double* isd, float* isf, int nX,
                                  cudaStream_t s);
cudaError_t launch_cut_to_float(const double* dp, float* fp, long long count, cudaStream_t s);
// apply records and node / enriched id quadruples of the cut tets (needs isD, phases, scale)
cudaError_t launch_cut_records(CutData cd, const double* isD, int nX, GridDev g, PhaseDev ph,
                               const float* scale, int4* n4, int4* e4, double* r64, float* r32,
                               cudaStream_t s);
// cached scaled element matrices of the cut tets (packed upper triangle, FP32; isD: D0^-1/2)
constexpr int kCutPacked = 24 * 25 / 2;
cudaError_t launch_cut_matrix(CutData cd, const double* isD, int nX, GridDev g, PhaseDev ph,
                              const float* scale, float* kc, cudaStream_t s);

// ---- stiffness apply (apply.cu)
struct ApplyArgs {
  GridDev g;
  PhaseDev ph;
  const uint16_t* code;
  const float* scale;      // per-voxel modulus scale or nullptr
  const double* eps;       // per RHS Mandel strain (n_rhs x 6) or nullptr (linear apply)
  const int* active;       // per RHS flag or nullptr (all active)
  long long stride;        // elements per RHS vector (3 (N + nX))
  int nX;
  double* partials;        // [rhs][7][nparts]: 0 = <d, A d>, 1..6 = int C eps (Mandel)
  int nparts;              // partial slots per RHS and component
  int part_offset_cut;     // first slot of the cut-tet kernel
  unsigned long long* units_uncut;  // optional counters of processed right-hand sides
  unsigned long long* units_cut;
  int want_sig;            // 1: partials carry int_e sigma:eps and int_e sigma (always with eps);
                           // 0: partial 0 is <d, q> and the stress integrals are 0
  // fused CG update in the stencil (standard DOFs): the operator is applied to
  // d_new = z + beta d_old (d_old = the kernel's input d), d_new is stored to fdnew and
  // u += alpha d_old at the block's own nodes; alpha and beta come from st[rhs]
  const void* fz;          // z (same type as d) or nullptr (no fused update)
  void* fdnew;
  void* fu;
  const RhsState* st;
  // FP32 cached cut-tet matrices (kCutPacked x ncut) or nullptr; used by the FP32 cut apply of
  // linear applies without stress integrals (the inner CG iterations)
  const float* kcache = nullptr;
  // launch shape of the cut-tet kernel (0: the defaults, apply_cut_blocks(ncut) blocks and up
  // to kCutMaxR right-hand sides per launch); the partial slots must hold cut_blocks
  int cut_blocks = 0;
  int cut_rpl = 0;
};
// T is the arithmetic type (float, double or dw = double-word on FP64 data); the vectors are
// stored as Store<T>::type
template <typename T>
cudaError_t launch_apply(const typename Store<T>::type* d, typename Store<T>::type* q,
                         const typename Store<T>::type* isD, CutData cd, const ApplyArgs& a,
                         int n_rhs, cudaStream_t s);
template <typename T>
cudaError_t launch_apply_uncut(const typename Store<T>::type* d, typename Store<T>::type* q,
                               const ApplyArgs& a, int n_rhs, cudaStream_t s);
template <typename T>
cudaError_t launch_apply_cut(const typename Store<T>::type* d, typename Store<T>::type* q,
                             const typename Store<T>::type* isD, CutData cd, const ApplyArgs& a,
                             int n_rhs, cudaStream_t s);
int apply_uncut_blocks(const GridDev& g);
int apply_cut_blocks(int ncut);      // the default grid of the cut-tet kernel
int apply_cut_blocks_max(int ncut);  // the largest grid a tuned launch shape may use

// per-voxel average stress of the (scaled) solution u, double
cudaError_t launch_voxel_stress(const double* u, const double* isD, CutData cd,
                                const ApplyArgs& a, double* out, int n_rhs, cudaStream_t s);

// ---- preconditioner (fft.cu)
struct FftPlan;  // opaque
FftPlan* fft_plan_create(const GridDev& g, cudaError_t* err);
void fft_plan_destroy(FftPlan* p);
size_t fft_spectrum_elems(const FftPlan* p);  // complex elements per RHS
// z = P^-1 f per RHS (std part via FFT + Green, enr part identity); f^T z partials into
// partials[rhs][nparts] (slots 0..nb-1).  spec: workspace of n_rhs * spectrum elems complex.
// With q != nullptr the first pass also applies f -= alpha q (alpha = st[rhs].alpha) and stores f.
// eblk (6 x nX, may be null): inverse 3x3 blocks of the block enriched preconditioner.
// group > 0: the FFT passes run `group` right-hand sides at a time (the spectrum of a group stays
// in L2 between the passes; the launch-shape tuner picks it); 0: all at once
template <typename T>
cudaError_t launch_precondition(const FftPlan* p, T* f, T* z, void* spec, long long stride,
                                int nX, const int* active, double* partials, int nparts,
                                int n_rhs, cudaStream_t s, unsigned long long* units = nullptr,
                                const T* q = nullptr, const RhsState* st = nullptr,
                                const T* eblk = nullptr, int group = 0);
// partial-sum slots written by one precondition call (FP64 or FP32 kernels)
int precondition_blocks(const FftPlan* p, int nX, bool dbl);

// ---- CG vector ops and scalar finalisation (cg.cu)
template <typename T>
cudaError_t launch_axpy_cg(T* u, T* f, const T* d, const T* q, const RhsState* st,
                           long long stride, int n_rhs, cudaStream_t s);
template <typename T>
cudaError_t launch_xpby(T* d, const T* z, const RhsState* st, long long stride, int n_rhs,
                        cudaStream_t s);
template <typename Tin, typename Tout>
cudaError_t launch_scale_copy(const Tin* x, Tout* y, double a, long long stride, int n_rhs,
                              const int* active, cudaStream_t s);
template <typename T>
cudaError_t launch_add_to_double(double* u, const T* dlt, long long stride, int n_rhs,
                                 const int* active, cudaStream_t s);
// enriched block of the fused CG update: d_new = z + beta d_old, u += alpha d_old on [off, stride)
template <typename T>
cudaError_t launch_cg_update_tail(const T* z, const T* dold, T* dnew, T* u, const RhsState* st,
                                  long long off, long long stride, int n_rhs, cudaStream_t s);
// the update u += alpha d still pending after the last iteration (all right-hand sides); d is
// dA or dB per right-hand side (RhsState::dpar)
template <typename T>
cudaError_t launch_cg_finish(T* u, const T* dA, const T* dB, const RhsState* st, long long stride,
                             int n_rhs, cudaStream_t s);
// mode: 0 = after the initial total apply (sig = partials 1..6), 1 = after an apply (alpha),
// 2 = after a preconditioner application (rr, beta, stopping rule), 3 = initial precond
struct FinArgs {
  int mode;
  int crit;        // 0: absolute-stress stopping rule, 1: relative rr reduction
  double tol;
  double volY;
  int maxit;
  int nparts;      // stride of the partial-sum rows
  int nparts_used; // valid partial sums per row
  // mode 3 of an FP64 residual check in iterative refinement: set the per-RHS relative target
  // of the next inner solve so that it aims at the outer tolerance (never below inner_floor)
  int set_rel;
  double inner_floor;
  int parity;      // buffer index of the direction used in this iteration (recorded on exit)
  // iteration scheme on the same operator: 0 linear CG (Algorithm 1), 1 basic scheme (fixed
  // step step0, steepest-descent directions), 2 Barzilai-Borwein (step = the previous Cauchy
  // step rr / <d, A d>, step0 first), 3 nonlinear CG (fixed step step0, Fletcher-Reeves momentum)
  int scheme;
  double step0;
  // Barzilai-Borwein step rule (scheme 2): 0 BB1 and 1 BB2 in the metric of P, 2 BB1 and BB2
  // alternating, 3 BB1 and 4 BB2 in the Euclidean metric of the scaled DOFs (these read
  // bbpart); the step is renewed every bb_cycle iterations and kept in between
  int bb_rule;
  int bb_cycle;
  const double* bbpart;  // [rhs][2][kBBParts]: <d, d> and <A d, A d> partial sums, or nullptr
  // mode 0: the stress integrals are sig_base[rhs] (a residual update) plus this apply's, or this
  // apply's alone (sig_base nullptr); they are also recorded in sig_keep[rhs] when given
  const double* sig_base;
  double* sig_keep;
};
constexpr int kBBParts = 256;
// <d, d> and <q, q> per right-hand side into part[rhs][2][kBBParts] (Euclidean BB steps)
template <typename T>
cudaError_t launch_bb_dots(const T* d, const T* q, const int* active, long long stride, int n_rhs,
                           double* part, cudaStream_t s);
// act[rhs] mirrors st[rhs].active for the kernels' early exit
cudaError_t launch_finalize(RhsState* st, const double* partials, FinArgs fa, int n_rhs, int* act,
                            cudaStream_t s);
cudaError_t launch_init_state(RhsState* st, int* act, int n_rhs, const int* mask, cudaStream_t s);

// ---- device-driven loops (loop.cu)
struct LoopState {
  unsigned long long t0;  // globaltimer at the loop's start
  unsigned rounds;        // body rounds run
  int timed_out;          // 1: the device-time limit ended the loop
};
// captures one round of a loop body on `stream` (called while the stream is capturing)
using LoopBody = std::function<cudaError_t(cudaStream_t stream)>;
// One device-driven loop of a graph: a start kernel, then a conditional while node whose body is
// one round (captured on `stream`) followed by the condition kernel: continue while some act[r],
// r < nr, is set, fewer than max_rounds rounds ran and less than limit_ns device time passed
// (limit_ns < 0: no limit).  act and st live in device memory.
struct LoopSpec {
  cudaStream_t stream;
  LoopBody body;
  const int* act;
  int nr;
  LoopState* st;
  unsigned max_rounds;
  long long limit_ns;
};
// An executable graph of independent loops (one per context; no dependencies between them).
cudaError_t build_loop_graph(const std::vector<LoopSpec>& loops, cudaGraphExec_t* exec);

// ---- gradient (grad.cu)
// values reduced per gradient call: dLoss/dlambda_p (p < kMaxPhases), dLoss/dmu_p, then the 21
// upper entries of the energy-form C_eff
constexpr int kGradValues = 2 * kMaxPhases + 21;
struct GradArgs {
  GridDev g;
  PhaseDev ph;
  const uint16_t* code;
  const float* scale;
  long long stride;
  int nX;
  double G[36];           // dLoss/dC_eff
  double* partials;       // [kGradValues][nparts]: dlam[3], dmu[3], C_energy upper triangle (21)
  int nparts;
  int part_offset_cut;
};
// hi, lo (6 * stride floats each, scratch): the mixed-precision solver's gradient (float pairs of U,
// strain products in FP32); nullptr: all FP64
cudaError_t launch_grad(const double* U, const double* isD, CutData cd, const GradArgs& a,
                        double* dscale, float* hi, float* lo, cudaStream_t s);
int grad_blocks_uncut(const GridDev& g);
int grad_blocks_cut(int ncut);
cudaError_t launch_reduce_partials(const double* partials, int nvals, int nparts, int ncount,
                                   double* out, cudaStream_t s);

}  // namespace xfft
