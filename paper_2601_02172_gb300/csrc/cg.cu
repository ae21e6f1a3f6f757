// Vector updates and FP64 scalar finalisation of the linear CG of Algorithm 1.
//
// Reading of Algorithm 1 (the printed sign of f - alpha z does not match r(u) = A u - b):
// f is the negative residual -b - A u, z = A d is the linear part of the residual map,
//   alpha = res^2 / <A d, d>,  u += alpha d,  f -= alpha A d,  z = P^{-1} f,
//   res_new^2 = f^T z,  beta = res_new^2 / res^2,  d = z + beta d,
// and the loop stops once sqrt(res^2 / |Y|) <= tol ||<sigma(u)>_Y|| (eqs. stoppingCriterion,
// convergence; dividing by |Y| makes both sides stresses).  <sigma(u)>_Y is tracked as
// sigma_int(u + alpha d) = sigma_int(u) + alpha int C grad^s d with the integral fused into the
// stiffness apply.  All scalars are FP64 and live on the device: one finalisation block per
// right-hand side reduces the per-block partial sums in a fixed order (deterministic).
#include <cuda_runtime.h>
#include <math.h>

#include "xfft_kernels.h"

namespace xfft {

template <typename T>
__global__ void k_axpy_cg(T* __restrict__ u, T* __restrict__ f, const T* __restrict__ d,
                          const T* __restrict__ q, const RhsState* __restrict__ st, long long stride) {
  const int rhs = blockIdx.y;
  if (!st[rhs].active) return;
  const T a = (T)st[rhs].alpha;
  T* ur = u + rhs * stride;
  T* fr = f + rhs * stride;
  const T* dr = d + rhs * stride;
  const T* qr = q + rhs * stride;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x) {
    ur[i] += a * dr[i];
    fr[i] -= a * qr[i];
  }
}

template <typename T>
__global__ void k_xpby(T* __restrict__ d, const T* __restrict__ z, const RhsState* __restrict__ st,
                       long long stride) {
  const int rhs = blockIdx.y;
  if (!st[rhs].active) return;
  const T b = (T)st[rhs].beta;
  T* dr = d + rhs * stride;
  const T* zr = z + rhs * stride;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x)
    dr[i] = zr[i] + b * dr[i];
}

template <typename Tin, typename Tout>
__global__ void k_scale_copy(const Tin* __restrict__ x, Tout* __restrict__ y, double a,
                             long long stride, const int* __restrict__ active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const Tin* xr = x + rhs * stride;
  Tout* yr = y + rhs * stride;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x)
    yr[i] = (Tout)(a * (double)xr[i]);
}

template <typename T>
__global__ void k_add_to_double(double* __restrict__ u, const T* __restrict__ dlt, long long stride,
                                const int* __restrict__ active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  double* ur = u + rhs * stride;
  const T* dr = dlt + rhs * stride;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x)
    ur[i] += (double)dr[i];
}

template <typename T>
__global__ void k_cg_update_tail(const T* __restrict__ z, const T* __restrict__ dold, T* __restrict__ dnew,
                                 T* __restrict__ u, const RhsState* __restrict__ st, long long off,
                                 long long stride) {
  const int rhs = blockIdx.y;
  if (!st[rhs].active) return;
  const T a = (T)st[rhs].alpha, b = (T)st[rhs].beta;
  const long long base = rhs * stride;
  for (long long i = off + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x) {
    const T d0 = dold[base + i];
    dnew[base + i] = z[base + i] + b * d0;
    u[base + i] += a * d0;
  }
}

template <typename T>
__global__ void k_cg_finish(T* __restrict__ u, const T* __restrict__ dA, const T* __restrict__ dB,
                            const RhsState* __restrict__ st, long long stride) {
  const int rhs = blockIdx.y;
  const T a = (T)st[rhs].alpha;
  if (a == T(0)) return;
  T* ur = u + rhs * stride;
  const T* dr = (st[rhs].dpar ? dB : dA) + rhs * stride;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x)
    ur[i] += a * dr[i];
}

static unsigned vec_blocks(long long stride) {
  long long nb = (stride + 255) / 256;
  if (nb > 2048) nb = 2048;
  return (unsigned)(nb < 1 ? 1 : nb);
}

template <typename T>
cudaError_t launch_axpy_cg(T* u, T* f, const T* d, const T* q, const RhsState* st, long long stride,
                           int n_rhs, cudaStream_t s) {
  k_axpy_cg<T><<<dim3(vec_blocks(stride), n_rhs), 256, 0, s>>>(u, f, d, q, st, stride);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xpby(T* d, const T* z, const RhsState* st, long long stride, int n_rhs,
                        cudaStream_t s) {
  k_xpby<T><<<dim3(vec_blocks(stride), n_rhs), 256, 0, s>>>(d, z, st, stride);
  return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_scale_copy(const Tin* x, Tout* y, double a, long long stride, int n_rhs,
                              const int* active, cudaStream_t s) {
  k_scale_copy<Tin, Tout><<<dim3(vec_blocks(stride), n_rhs), 256, 0, s>>>(x, y, a, stride, active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_to_double(double* u, const T* dlt, long long stride, int n_rhs,
                                 const int* active, cudaStream_t s) {
  k_add_to_double<T><<<dim3(vec_blocks(stride), n_rhs), 256, 0, s>>>(u, dlt, stride, active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update_tail(const T* z, const T* dold, T* dnew, T* u, const RhsState* st,
                                  long long off, long long stride, int n_rhs, cudaStream_t s) {
  if (stride <= off) return cudaSuccess;
  k_cg_update_tail<T><<<dim3(vec_blocks(stride - off), n_rhs), 256, 0, s>>>(z, dold, dnew, u, st, off, stride);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_finish(T* u, const T* dA, const T* dB, const RhsState* st, long long stride,
                             int n_rhs, cudaStream_t s) {
  k_cg_finish<T><<<dim3(vec_blocks(stride), n_rhs), 256, 0, s>>>(u, dA, dB, st, stride);
  return cudaGetLastError();
}

template cudaError_t launch_cg_update_tail<float>(const float*, const float*, float*, float*,
                                                  const RhsState*, long long, long long, int, cudaStream_t);
template cudaError_t launch_cg_update_tail<double>(const double*, const double*, double*, double*,
                                                   const RhsState*, long long, long long, int, cudaStream_t);
template cudaError_t launch_cg_finish<float>(float*, const float*, const float*, const RhsState*,
                                             long long, int, cudaStream_t);
template cudaError_t launch_cg_finish<double>(double*, const double*, const double*, const RhsState*,
                                              long long, int, cudaStream_t);
template cudaError_t launch_axpy_cg<float>(float*, float*, const float*, const float*,
                                           const RhsState*, long long, int, cudaStream_t);
template cudaError_t launch_axpy_cg<double>(double*, double*, const double*, const double*,
                                            const RhsState*, long long, int, cudaStream_t);
template cudaError_t launch_xpby<float>(float*, const float*, const RhsState*, long long, int,
                                        cudaStream_t);
template cudaError_t launch_xpby<double>(double*, const double*, const RhsState*, long long, int,
                                         cudaStream_t);
template cudaError_t launch_scale_copy<double, double>(const double*, double*, double, long long,
                                                       int, const int*, cudaStream_t);
template cudaError_t launch_scale_copy<double, float>(const double*, float*, double, long long,
                                                      int, const int*, cudaStream_t);
template cudaError_t launch_scale_copy<float, double>(const float*, double*, double, long long,
                                                      int, const int*, cudaStream_t);
template cudaError_t launch_scale_copy<float, float>(const float*, float*, double, long long, int,
                                                     const int*, cudaStream_t);
template cudaError_t launch_add_to_double<float>(double*, const float*, long long, int,
                                                 const int*, cudaStream_t);
template cudaError_t launch_add_to_double<double>(double*, const double*, long long, int,
                                                  const int*, cudaStream_t);

// <d, d> and <q, q> per right-hand side (Euclidean Barzilai-Borwein steps): kBBParts blocks
// per right-hand side write their partial sums, the finalisation adds them in a fixed order
template <typename T>
__global__ void k_bb_dots(const T* __restrict__ d, const T* __restrict__ q, const int* __restrict__ active,
                          long long stride, double* __restrict__ part) {
  __shared__ double red[2 * 32];
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;  // uniform per block
  const T* dr = d + rhs * stride;
  const T* qr = q + rhs * stride;
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride;
       i += (long long)gridDim.x * blockDim.x) {
    const double x = (double)dr[i], y = (double)qr[i];
    v[0] += x * x;
    v[1] += y * y;
  }
  double tot[2];
  block_sum<2>(v, red, tot);
  if (threadIdx.x == 0) {
    part[((long long)rhs * 2 + 0) * kBBParts + blockIdx.x] = tot[0];
    part[((long long)rhs * 2 + 1) * kBBParts + blockIdx.x] = tot[1];
  }
}

template <typename T>
cudaError_t launch_bb_dots(const T* d, const T* q, const int* active, long long stride, int n_rhs,
                           double* part, cudaStream_t s) {
  k_bb_dots<T><<<dim3(kBBParts, n_rhs), 256, 0, s>>>(d, q, active, stride, part);
  return cudaGetLastError();
}
template cudaError_t launch_bb_dots<float>(const float*, const float*, const int*, long long, int,
                                           double*, cudaStream_t);
template cudaError_t launch_bb_dots<double>(const double*, const double*, const int*, long long, int,
                                            double*, cudaStream_t);

// ---------------------------------------------------------------- finalisation
__device__ inline bool stop_rule(const RhsState& s, const FinArgs& fa) {
  if (!(s.rr > 0.0)) return true;
  if (fa.crit == 1) {
    const double rel = s.rel > 0.0 ? s.rel : fa.tol;
    return s.rr <= rel * rel * s.rr0;
  }
  double sn = 0.0;
  for (int k = 0; k < 6; ++k) sn += s.sig[k] * s.sig[k];
  return sqrt(s.rr / fa.volY) <= fa.tol * sqrt(sn) / fa.volY;
}

__global__ void k_finalize(RhsState* __restrict__ st, int* __restrict__ act,
                           const double* __restrict__ partials, FinArgs fa, int ncount) {
  __shared__ double red[7 * 32];
  const int rhs = blockIdx.x;
  RhsState& s = st[rhs];
  if (!s.active) return;  // uniform per block
  const int nv = (fa.mode <= 1) ? 7 : 1;  // values per RHS in the partial rows
  // an iteration under the relative stopping rule (crit 1) needs <d, A d> alone: the stress
  // increments (zero there) are not read
  const int nread = (fa.mode == 1 && fa.crit == 1) ? 1 : nv;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < ncount; i += blockDim.x)
    for (int k = 0; k < nread; ++k) v[k] += partials[((long long)rhs * nv + k) * fa.nparts + i];
  double tot[7];
  block_sum<7>(v, red, tot);
  if (threadIdx.x != 0) return;
  if (fa.mode == 0) {
    for (int k = 0; k < 6; ++k) s.sig[k] = (fa.sig_base ? fa.sig_base[6 * rhs + k] : 0.0) + tot[1 + k];
    if (fa.sig_keep)
      for (int k = 0; k < 6; ++k) fa.sig_keep[6 * rhs + k] = s.sig[k];
  } else if (fa.mode == 1) {
    const double dq_prev = s.dq;
    s.dq = tot[0];
    for (int k = 0; k < 6; ++k) s.sd[k] = tot[1 + k];
    const double a = s.rr / s.dq;
    if (!(s.dq > 0.0) || !isfinite(a)) {
      s.status = 5;
      s.active = 0;
      s.alpha = 0.0;
      s.dpar = fa.parity;
    } else {
      // 0 CG: exact line search; 1 basic and 3 nonlinear CG: fixed step s0; 2 BB: a step from
      // the previous iteration's differences du = s d, dg = s A d (steepest-descent directions
      // d = P^-1 f), s0 first
      double step = a;
      if (fa.scheme == 1 || fa.scheme == 3) {
        step = fa.step0;
      } else if (fa.scheme == 2) {
        double dd = 0.0, qq = 0.0;
        if (fa.bbpart) {  // (thread 0 only from here on) fixed-order sum of the block partials
          for (int i = 0; i < kBBParts; ++i) {
            dd += fa.bbpart[((long long)rhs * 2 + 0) * kBBParts + i];
            qq += fa.bbpart[((long long)rhs * 2 + 1) * kBBParts + i];
          }
        }
        if (s.iters == 0) {
          step = fa.step0;
        } else if (fa.bb_cycle > 1 && (s.iters - 1) % fa.bb_cycle != 0) {
          step = s.bb_step;  // cyclic rule: keep the step of the cycle
        } else {
          const double sp = s.alpha;  // previous step
          // BB1 in the P metric: <du, P du> / <du, dg> = rr_prev / <d, A d>_prev (the previous
          // exact line-search step); BB2 in the P metric: <du, dg> / <dg, P^-1 dg> with
          // <dg, P^-1 dg> = rr - rr_prev + 2 s <d, A d>_prev (d = P^-1 f_prev)
          const double bb1 = s.cauchy;
          const double den2 = s.rr - s.rr_prev + 2.0 * sp * dq_prev;
          const double bb2 = sp * sp * dq_prev / den2;
          const double bb1e = s.dd / dq_prev, bb2e = dq_prev / s.qq;
          const int rule = fa.bb_rule == 2 ? ((s.iters & 1) ? 1 : 0) : fa.bb_rule;  // BB2 on odd
          step = rule == 0 ? bb1 : rule == 1 ? bb2 : rule == 3 ? bb1e : bb2e;
          if (!(step > 0.0) || !isfinite(step)) step = bb1;  // safeguard: BB1 is positive
        }
        s.bb_step = step;
        s.dd = dd;
        s.qq = qq;
      }
      s.cauchy = a;
      s.alpha = step;
      for (int k = 0; k < 6; ++k) s.sig[k] += step * s.sd[k];
    }
  } else {
    const double rr = tot[0];
    if (!isfinite(rr)) {
      s.status = 5;
      s.active = 0;
    } else if (fa.mode == 3) {
      s.rr = rr;
      s.rr0 = rr;
      s.beta = 0.0;
      if (stop_rule(s, fa)) {
        s.converged = 1;
        s.active = 0;
      } else if (fa.set_rel) {
        // the inner solve should bring sqrt(rr/|Y|) to half the outer target
        double sn = 0.0;
        for (int k = 0; k < 6; ++k) sn += s.sig[k] * s.sig[k];
        const double target = 0.5 * fa.tol * sqrt(sn) / fa.volY;
        const double res = sqrt(rr / fa.volY);
        double rel = res > 0.0 ? target / res : 1.0;
        if (rel < fa.inner_floor) rel = fa.inner_floor;
        if (rel > 0.5) rel = 0.5;
        s.rel = rel;
      }
    } else {
      // Fletcher-Reeves momentum for linear and nonlinear CG; basic and BB: steepest descent
      s.beta = ((fa.scheme == 0 || fa.scheme == 3) && s.rr > 0.0) ? rr / s.rr : 0.0;
      s.rr_prev = s.rr;
      s.rr = rr;
      s.iters += 1;
      s.dpar = fa.parity;
      if (stop_rule(s, fa)) {
        s.converged = 1;
        s.active = 0;
      } else if (s.iters >= fa.maxit) {
        s.status = 4;
        s.active = 0;
      }
    }
  }
  act[rhs] = s.active;
}

cudaError_t launch_finalize(RhsState* st, const double* partials, FinArgs fa, int n_rhs, int* act,
                            cudaStream_t s) {
  k_finalize<<<n_rhs, 512, 0, s>>>(st, act, partials, fa, fa.nparts_used);
  return cudaGetLastError();
}

__global__ void k_init_state(RhsState* st, int* act, int n_rhs, const int* mask) {
  const int r = threadIdx.x;
  if (r >= n_rhs) return;
  RhsState s;
  s.rr = s.rr0 = s.dq = s.alpha = s.beta = s.rel = s.cauchy = 0.0;
  s.rr_prev = s.dd = s.qq = s.bb_step = 0.0;
  for (int k = 0; k < 6; ++k) s.sig[k] = s.sd[k] = 0.0;
  s.active = mask ? mask[r] : 1;
  s.dpar = 0;
  s.iters = 0;
  s.status = 0;
  s.converged = 0;
  st[r] = s;
  act[r] = s.active;
}

cudaError_t launch_init_state(RhsState* st, int* act, int n_rhs, const int* mask, cudaStream_t s) {
  k_init_state<<<1, 64, 0, s>>>(st, act, n_rhs, mask);
  return cudaGetLastError();
}

}  // namespace xfft
