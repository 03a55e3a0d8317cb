// Volume integral equation of an inhomogeneous medium (Section 7, Eqs. 7.1-7.5):
//   p(x) - int G_{k_n}(x - y) q(y) p(y) dy = b(x),   q(y) = k_n(y)^2 - kbar_n^2,
// discretised with the quadrature of vp_apply, (I - V_{k_n} Q) p = b, and solved by
// BiCGStab.  Each iteration applies the operator twice (a pointwise product with q and
// one vp_apply each); inner products are accumulated in FP64 on the device and the
// scalar recurrences run on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>

#include "vp.h"
#include "vp_internal.cuh"

namespace {

using cplx = std::complex<double>;

struct Vie {
  vp_plan_t plan;
  long long n;
  const float2* q;
  float2* tmp;    // q * x
  float2* u;      // V[q x]
  double* acc;    // 2 doubles on the device
  cudaStream_t s;
};

int cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return VP_OK;
  if (e == cudaErrorMemoryAllocation) return VP_ERR_NOMEM;
  return VP_ERR_CUDA;
}

// y = x - V[q x]
int apply_op(Vie& v, const float2* x, float2* y) {
  cudaError_t e = vp::launch_mul(v.n, v.q, x, v.tmp, v.s);
  if (e != cudaSuccess) return cuda_st(e);
  int st = vp_apply(v.plan, v.tmp, v.u, v.s);
  if (st != VP_OK) return st;
  return cuda_st(vp::launch_axpby(v.n, make_float2(1.f, 0.f), x, make_float2(-1.f, 0.f), v.u, y, v.s));
}

int dot(Vie& v, const float2* x, const float2* y, cplx& out) {
  cudaError_t e = vp::launch_dot(v.n, x, y, 1, v.acc, v.s);
  double h[2];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, v.acc, sizeof(h), cudaMemcpyDeviceToHost, v.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.s);
  if (e != cudaSuccess) return cuda_st(e);
  out = cplx(h[0], h[1]);
  return VP_OK;
}

int axpby(Vie& v, cplx a, const float2* x, cplx b, const float2* y, float2* out) {
  return cuda_st(vp::launch_axpby(v.n, make_float2((float)a.real(), (float)a.imag()), x,
                                  make_float2((float)b.real(), (float)b.imag()), y, out, v.s));
}

}  // namespace

extern "C" {

VP_API int vp_vie_solve(vp_plan_t plan, const void* q, const void* b, void* x, double tol, int max_iter,
                        int* iters, double* relres, vp_stream_t stream) {
  if (!plan || !q || !b || !x || !(tol > 0) || max_iter < 1) return VP_ERR_ARG;
  vp_plan_info info;
  int st = vp_plan_get_info(plan, &info);
  if (st != VP_OK) return st;
  if (!info.khat_ready) return VP_ERR_STATE;
  Vie v;
  v.plan = plan;
  v.n = (long long)info.n[0] * info.n[1] * info.n[2];
  v.q = (const float2*)q;
  v.s = (cudaStream_t)stream;
  const float2* B = (const float2*)b;
  float2* X = (float2*)x;
  // workspace: r, rh, p, w (= A p), s, t, tmp, u and two doubles
  const size_t vec = (size_t)v.n * sizeof(float2);
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, 8 * vec + 256, v.s);
  if (e != cudaSuccess) return cuda_st(e);
  float2* r = (float2*)base;
  float2* rh = (float2*)(base + vec);
  float2* p = (float2*)(base + 2 * vec);
  float2* w = (float2*)(base + 3 * vec);
  float2* sv = (float2*)(base + 4 * vec);
  float2* t = (float2*)(base + 5 * vec);
  v.tmp = (float2*)(base + 6 * vec);
  v.u = (float2*)(base + 7 * vec);
  v.acc = (double*)(base + 8 * vec);
  int it = 0;
  double res = 0.0;
  do {
    cplx bb;
    if ((st = dot(v, B, B, bb)) != VP_OK) break;
    const double bnorm = std::sqrt(bb.real());
    if (bnorm == 0.0) {  // b = 0: x = 0
      st = cuda_st(cudaMemsetAsync(X, 0, vec, v.s));
      res = 0.0;
      break;
    }
    // r = b - A x,  rh = r,  p = w = 0
    if ((st = apply_op(v, X, w)) != VP_OK) break;
    if ((st = axpby(v, 1.0, B, -1.0, w, r)) != VP_OK) break;
    if ((st = cuda_st(cudaMemcpyAsync(rh, r, vec, cudaMemcpyDeviceToDevice, v.s))) != VP_OK) break;
    if ((st = cuda_st(cudaMemsetAsync(p, 0, vec, v.s))) != VP_OK) break;
    if ((st = cuda_st(cudaMemsetAsync(w, 0, vec, v.s))) != VP_OK) break;
    cplx rr;
    if ((st = dot(v, r, r, rr)) != VP_OK) break;
    res = std::sqrt(rr.real()) / bnorm;
    cplx rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    while (res > tol && it < max_iter) {
      cplx rho;
      if ((st = dot(v, rh, r, rho)) != VP_OK) break;
      if (std::abs(rho) == 0.0) break;  // breakdown: return the current iterate
      const cplx beta = (rho / rho_prev) * (alpha / omega);
      // p = r + beta (p - omega w)
      if ((st = axpby(v, 1.0, p, -omega, w, p)) != VP_OK) break;
      if ((st = axpby(v, 1.0, r, beta, p, p)) != VP_OK) break;
      if ((st = apply_op(v, p, w)) != VP_OK) break;
      cplx rhw;
      if ((st = dot(v, rh, w, rhw)) != VP_OK) break;
      if (std::abs(rhw) == 0.0) break;
      alpha = rho / rhw;
      // s = r - alpha w
      if ((st = axpby(v, 1.0, r, -alpha, w, sv)) != VP_OK) break;
      ++it;
      cplx ss;
      if ((st = dot(v, sv, sv, ss)) != VP_OK) break;
      if (std::sqrt(ss.real()) / bnorm <= tol) {
        if ((st = axpby(v, 1.0, X, alpha, p, X)) != VP_OK) break;
        res = std::sqrt(ss.real()) / bnorm;
        break;
      }
      if ((st = apply_op(v, sv, t)) != VP_OK) break;
      cplx ts, tt;
      if ((st = dot(v, t, sv, ts)) != VP_OK) break;
      if ((st = dot(v, t, t, tt)) != VP_OK) break;
      omega = tt.real() > 0 ? ts / tt.real() : cplx(0.0);
      // x = x + alpha p + omega s;  r = s - omega t
      if ((st = axpby(v, 1.0, X, alpha, p, X)) != VP_OK) break;
      if ((st = axpby(v, 1.0, X, omega, sv, X)) != VP_OK) break;
      if ((st = axpby(v, 1.0, sv, -omega, t, r)) != VP_OK) break;
      if ((st = dot(v, r, r, rr)) != VP_OK) break;
      res = std::sqrt(rr.real()) / bnorm;
      rho_prev = rho;
      if (std::abs(omega) == 0.0) break;
    }
  } while (false);
  cudaError_t ef = cudaFreeAsync(base, v.s);
  if (st == VP_OK && ef != cudaSuccess) st = cuda_st(ef);
  if (iters) *iters = it;
  if (relres) *relres = res;
  return st;
}

}  // extern "C"
