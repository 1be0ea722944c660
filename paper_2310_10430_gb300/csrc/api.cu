// C ABI of the parallel-in-time Biot solver (include/biot_pint.h).
//
// Host-side orchestration only: argument checks, device memory, the window
// schedule of the inverted time stepping (Alg. 3 as snapshot sweeps), and data
// exchange. Every arithmetic step of the method runs in the kernels of
// assembly.cu, spmm.cu, band.cu and krylov.cu.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <new>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>

namespace biot {

std::atomic<int64_t> g_launches{0};
int krylov_record_doubles();

namespace {
thread_local std::string g_create_error = "no error";
}

biot_status fail(biot_ctx* ctx, biot_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_error = buf;
  return st;
}

biot_status cuda_check(biot_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BIOT_OK;
  return fail(ctx, e == cudaErrorMemoryAllocation ? BIOT_E_OOM : BIOT_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

biot_status dalloc(biot_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? BIOT_E_OOM : BIOT_E_CUDA, "cudaMalloc(%zu): %s", bytes,
                cudaGetErrorString(e));
  }
  ctx->allocs.push_back(*p);
  ctx->alloc_bytes.push_back(bytes);
  ctx->device_bytes += (int64_t)bytes;
  return BIOT_OK;
}

void dfree(biot_ctx* ctx, void* p) {
  if (!p) return;
  for (size_t k = 0; k < ctx->allocs.size(); ++k)
    if (ctx->allocs[k] == p) {
      cudaFree(p);
      ctx->device_bytes -= (int64_t)ctx->alloc_bytes[k];
      ctx->allocs.erase(ctx->allocs.begin() + k);
      ctx->alloc_bytes.erase(ctx->alloc_bytes.begin() + k);
      return;
    }
}

void dfree_all(biot_ctx* ctx) {
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->alloc_bytes.clear();
  ctx->device_bytes = 0;
}

static size_t next_event(biot_ctx* ctx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_used++;
}

KTimer::KTimer(biot_ctx* c, int k) : ctx(c), kc(k) {
  if (!ctx->timing) return;
  a = next_event(ctx);
  if (a != (size_t)-1) cudaEventRecord(ctx->ev_pool[a], ctx->stream);
}

KTimer::~KTimer() {
  if (!ctx->timing || a == (size_t)-1) return;
  size_t b = next_event(ctx);
  if (b == (size_t)-1) return;
  cudaEventRecord(ctx->ev_pool[b], ctx->stream);
  ctx->ev_marks[kc].emplace_back(a, b);
}

namespace {

// Tiled transposes between the device layout [dof][ld] (time fastest) and the
// host layout [step][n_dof] (FP64 staging). Optional row scale: divide on the way
// out, multiply on the way in.
template <typename S>
__global__ void k_dof_to_step(const S* __restrict__ src, int lds, int col0, int ncols, int nrows,
                              const double* __restrict__ rowscale, double* __restrict__ dst) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.x * 32, cb = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k, c = cb + threadIdx.x;
    double v = 0.0;
    if (r < nrows && c < ncols) {
      v = (double)src[(size_t)r * lds + col0 + c];
      if (rowscale) v /= rowscale[r];
    }
    tile[k][threadIdx.x] = v;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int c = cb + k, r = r0 + threadIdx.x;
    if (r < nrows && c < ncols) dst[(size_t)c * nrows + r] = tile[threadIdx.x][k];
  }
}

template <typename D>
__global__ void k_step_to_dof(const double* __restrict__ src, int ncols, int nrows, const double* __restrict__ rowscale,
                              D* __restrict__ dst, int ldd, int col0) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.x * 32, cb = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int c = cb + k, r = r0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < nrows && c < ncols) ? src[(size_t)c * nrows + r] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k, c = cb + threadIdx.x;
    if (r < nrows && c < ncols) {
      double v = tile[threadIdx.x][k];
      if (rowscale) v *= rowscale[r];
      dst[(size_t)r * ldd + col0 + c] = (D)v;
    }
  }
}

__global__ void k_cvt_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = (float)src[k];
}

__global__ void k_cvt_bf16(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = __double2bfloat16(src[k]);
}

// |D^{-1/2} f_ST|^2 contributions per step n (f_ST = f^n, plus A' x0 for n = 1).
__global__ void k_fst_norms(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
                            const int32_t* __restrict__ rowptr, const double* __restrict__ val,
                            const double* __restrict__ apval, const double* __restrict__ dsc,
                            const double* __restrict__ X, const double* __restrict__ F, int ldx, int lo, int ncols,
                            double* __restrict__ part, int ldp) {
  __shared__ double sm[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nn + gridDim.x - 1) / gridDim.x;
  const int vb = blockIdx.x * per, ve = min(nn, vb + per);
  for (int cb = 0; cb < ncols; cb += 32) {
    const int c = cb + lane;
    const bool cv = c < ncols;
    const int tn = lo + (cv ? c : 0);
    double acc = 0.0;
    for (int v = vb + warp; v < ve; v += 8) {
      double b2 = F[(size_t)(3 * v + 2) * ldx + tn];
      if (tn == 1) {
        const int32_t np = nodeptr[v];
        const int deg = nodeptr[v + 1] - np;
        const int32_t r2 = rowptr[3 * v] + 6 * deg;
        for (int k = 0; k < deg; ++k) {
          const int m = nbr[np + k];
          b2 += val[r2 + 3 * k] * X[(size_t)(3 * m) * ldx] + val[r2 + 3 * k + 1] * X[(size_t)(3 * m + 1) * ldx] +
                apval[np + k] * X[(size_t)(3 * m + 2) * ldx];
        }
      }
      const double p0 = dsc[3 * v] * F[(size_t)(3 * v) * ldx + tn];
      const double p1 = dsc[3 * v + 1] * F[(size_t)(3 * v + 1) * ldx + tn];
      const double p2 = dsc[3 * v + 2] * b2;
      if (cv) acc += p0 * p0 + p1 * p1 + p2 * p2;
    }
    sm[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && cv) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += sm[w][lane];
      part[(size_t)blockIdx.x * ldp + c] = s;
    }
    __syncthreads();
  }
}

bool bad_ctx(const biot_ctx* ctx) { return ctx == nullptr; }

biot_status need_assembled(biot_ctx* ctx) {
  if (!ctx->assembled) return fail(ctx, BIOT_E_STATE, "biot_assemble has not been called");
  return BIOT_OK;
}

biot_status need_precond(biot_ctx* ctx) {
  BIOT_TRY(need_assembled(ctx));
  if (ctx->precond == 0) return fail(ctx, BIOT_E_STATE, "biot_precond_setup has not been called");
  return BIOT_OK;
}

biot_status check_window(biot_ctx* ctx, int lo, int hi) {
  if (lo < 1 || hi > ctx->n_t || lo > hi)
    return fail(ctx, BIOT_E_INVALID, "window [%d, %d] outside 1..%d", lo, hi, ctx->n_t);
  if (hi - lo + 1 > ctx->wcap)
    return fail(ctx, BIOT_E_INVALID, "window of %d steps exceeds the work buffers (%d)", hi - lo + 1, ctx->wcap);
  return BIOT_OK;
}

// Residual of steps lo..lo+ncols-1 into V_0 (equilibrated), |d r|^2 and |d b|^2 into the
// column scalars; optionally the relative residuals to the host.
biot_status residual_window(biot_ctx* ctx, int lo, int ncols, double* rel_host) {
  launch_residual(ctx, lo, ncols, ctx->V, ctx->wcap);
  reduce_partials(ctx, 2, ncols, ctx->colscal + CS_RR * ctx->wcap, ctx->wcap, 0);
  BIOT_CU(ctx, cudaGetLastError());
  if (rel_host) {
    std::vector<double> rb(2 * (size_t)ctx->wcap);
    BIOT_CU(ctx, cudaMemcpyAsync(rb.data(), ctx->colscal, sizeof(double) * 2 * ctx->wcap, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < ncols; ++c) {
      const double rr = std::sqrt(rb[c]), bb = std::sqrt(rb[ctx->wcap + c]);
      rel_host[c] = bb > 0.0 ? rr / bb : (rr == 0.0 ? 0.0 : INFINITY);
    }
  }
  return BIOT_OK;
}

// Reduced-precision sweep: FP64 true residual of the window into the FP32 lp.V, FP64 relative norms.
biot_status residual_window_lp(biot_ctx* ctx, int lo, int ncols, double* rel_host) {
  launch_residual_lp(ctx, lo, ncols);
  reduce_partials(ctx, 2, ncols, ctx->colscal + CS_RR * ctx->wcap, ctx->wcap, 0);
  BIOT_CU(ctx, cudaGetLastError());
  if (rel_host) {
    std::vector<double> rb(2 * (size_t)ctx->wcap);
    BIOT_CU(ctx, cudaMemcpyAsync(rb.data(), ctx->colscal, sizeof(double) * 2 * ctx->wcap, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < ncols; ++c) {
      const double rr = std::sqrt(rb[c]), bb = std::sqrt(rb[ctx->wcap + c]);
      rel_host[c] = bb > 0.0 ? rr / bb : (rr == 0.0 ? 0.0 : INFINITY);
    }
  }
  return BIOT_OK;
}

// |D^{-1/2} f_ST|^2 summed over all steps.
biot_status fst_norm2(biot_ctx* ctx, double* out);

biot_status fst_norm2(biot_ctx* ctx, double* out) {
  double den = 0.0;
  std::vector<double> rb(ctx->wcap);
  for (int lo = 1; lo <= ctx->n_t; lo += ctx->wcap) {
    const int nc = std::min(ctx->wcap, ctx->n_t - lo + 1);
    BIOT_LAUNCH(k_fst_norms, kRedBlocks, 256, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr, ctx->nbr, ctx->rowptr,
                ctx->val, ctx->apval, ctx->dsc, ctx->X, ctx->F, ctx->ldx, lo, nc, ctx->part, ctx->wcap);
    reduce_partials(ctx, 1, nc, ctx->colscal + CS_BB * ctx->wcap, ctx->wcap, 0);
    BIOT_CU(ctx, cudaMemcpyAsync(rb.data(), ctx->colscal + CS_BB * ctx->wcap, sizeof(double) * nc,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < nc; ++c) den += rb[c];
  }
  *out = den;
  return BIOT_OK;
}

biot_status spacetime_residual(biot_ctx* ctx, double* out) {
  double num = 0.0, den = 0.0;
  std::vector<double> rb(ctx->wcap);
  for (int lo = 1; lo <= ctx->n_t; lo += ctx->wcap) {
    const int nc = std::min(ctx->wcap, ctx->n_t - lo + 1);
    launch_residual(ctx, lo, nc, ctx->V, ctx->wcap);
    reduce_partials(ctx, 1, nc, ctx->colscal + CS_RR * ctx->wcap, ctx->wcap, 0);
    BIOT_CU(ctx, cudaMemcpyAsync(rb.data(), ctx->colscal + CS_RR * ctx->wcap, sizeof(double) * nc,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < nc; ++c) num += rb[c];
  }
  BIOT_TRY(fst_norm2(ctx, &den));
  *out = den > 0.0 ? std::sqrt(num / den) : std::sqrt(num);
  return BIOT_OK;
}

bool low_precision(const biot_ctx* ctx) { return ctx->prm.precision != BIOT_FP64; }

std::map<std::string, int> read_tune_cache(const char* path) {
  std::map<std::string, int> out;
  if (!path) return out;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t k0 = line.find("\"key\": \"");
    const size_t v0 = line.find("\"variant\": ");
    if (k0 == std::string::npos || v0 == std::string::npos) continue;
    const size_t ks = k0 + 8, ke = line.find('"', ks);
    if (ke == std::string::npos) continue;
    out[line.substr(ks, ke - ks)] = std::atoi(line.c_str() + v0 + 11);
  }
  return out;
}

void write_tune_cache(const char* path, const std::map<std::string, int>& m) {
  if (!path) return;
  std::ofstream f(path);
  f << "{\"band_solve_variants\": [\n";
  size_t k = 0;
  for (const auto& kv : m)
    f << "  {\"key\": \"" << kv.first << "\", \"variant\": " << kv.second << "}" << (++k < m.size() ? "," : "")
      << "\n";
  f << "]}\n";
}

std::string tune_key(bool fp64, int N, int b, int ncols) {
  std::ostringstream o;
  o << (fp64 ? "fp64" : "fp32") << ":N" << N << ":b" << b << ":w" << ncols;
  return o.str();
}

biot_status device_status(biot_ctx* ctx) {
  int32_t st = 0;
  BIOT_CU(ctx, cudaMemcpyAsync(&st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  if (st != 0) return fail(ctx, BIOT_E_TIMEOUT, "a bounded device wait ran out (band-row bulk copy)");
  return BIOT_OK;
}



biot_status sweep_impl(biot_ctx* ctx, int lo, int hi, double* rel_out) {
  const int ncols = hi - lo + 1;
  if (low_precision(ctx)) {
    BIOT_TRY(residual_window_lp(ctx, lo, ncols, rel_out));
    return fgmres_cycle<float>(ctx, lo, 0, ncols);
  }
  BIOT_TRY(residual_window(ctx, lo, ncols, rel_out));
  return fgmres_cycle<double>(ctx, lo, 0, ncols);
}

// Tol-schedule PinT solve (Alg. 3 as snapshot sweeps, reading A5). T is the Krylov
// precision: double (plain FP64), or float (the cycle runs in FP32 on the correction
// of the FP64 residual and is added to the FP64 state). The residual and the
// retirement test are FP64 in both. A step active for stall_cap sweeps (0: never)
// retires as it is.
template <typename T>
biot_status tol_schedule(biot_ctx* ctx, double tol, int max_sweeps, int stall_cap, int* sweeps, bool* converged) {
  const int n_t = ctx->n_t;
  std::vector<double> rel(ctx->wcap);
  int lo = 1, w = 0, lo_since = 0;
  double first = -1.0;
  *converged = false;
  while (lo <= n_t) {
    if (w >= max_sweeps) {
      *sweeps = w;
      return BIOT_OK;
    }
    ++w;
    // causal start: step n becomes active at sweep n; eager start: every step from sweep 1
    const int top = ctx->prm.schedule == BIOT_SCHED_EAGER ? n_t : std::min(w, n_t);
    const int hi = std::min(top, lo + ctx->wcap - 1);
    const int nc = hi - lo + 1;
    if (sizeof(T) == 8) BIOT_TRY(residual_window(ctx, lo, nc, rel.data()));
    else BIOT_TRY(residual_window_lp(ctx, lo, nc, rel.data()));
    // a timed-out device wait leaves partial solves behind: report it before the divergence it causes
    for (int c = 0; c < nc; ++c)
      if (!std::isfinite(rel[c])) {
        BIOT_TRY(device_status(ctx));
        return fail(ctx, BIOT_E_DIVERGED, "non-finite residual at step %d, sweep %d", lo + c, w);
      }
    if (first < 0.0) first = rel[0];
    if (first > 0.0 && rel[0] > 1e6 * std::max(first, 1.0)) {
      BIOT_TRY(device_status(ctx));
      return fail(ctx, BIOT_E_DIVERGED, "residual of step %d grew to %.3g", lo, rel[0]);
    }
    int k = 0;
    while (k < nc && (rel[k] <= tol || (k == 0 && stall_cap > 0 && w - lo_since >= stall_cap))) ++k;
    BIOT_TRY(fgmres_cycle<T>(ctx, lo, k, nc - k));
    if (k > 0) lo_since = w;
    lo += k;
  }
  *sweeps = w;
  *converged = true;
  return BIOT_OK;
}

// Work buffers sized by N_t, the window capacity, n_iter and the precision.
biot_status alloc_time_buffers(biot_ctx* ctx) {
  const size_t nd = ctx->n_dof, wc = ctx->wcap, ld = ctx->ldx, nn = ctx->n_nodes;
  const bool lp = low_precision(ctx);
  BIOT_TRY(dalloc(ctx, (void**)&ctx->X, sizeof(double) * nd * ld));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->F, sizeof(double) * nd * ld));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->V, sizeof(double) * nd * wc * (lp ? 1 : ctx->n_iter + 1)));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->Wv, sizeof(double) * nd * wc));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->part, sizeof(double) * kPartBlocks * (kMaxIter + 2) * wc));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->colscal, sizeof(double) * kColScalars * wc));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->H, sizeof(double) * krylov_record_doubles() * wc));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->hvec, sizeof(double) * 2 * (kMaxIter + 1) * wc));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->kcol, sizeof(int32_t) * wc));
  if (!lp) {
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Z, sizeof(double) * nd * wc * ctx->n_iter));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->tu, sizeof(double) * 2 * nn * wc));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->tp, sizeof(double) * nn * wc));
    return BIOT_OK;
  }
  LowPrec& L = ctx->lp;
  BIOT_TRY(dalloc(ctx, (void**)&L.V, sizeof(float) * nd * wc * (ctx->n_iter + 1)));
  BIOT_TRY(dalloc(ctx, (void**)&L.Z, sizeof(float) * nd * wc * ctx->n_iter));
  BIOT_TRY(dalloc(ctx, (void**)&L.Wv, sizeof(float) * nd * wc));
  BIOT_TRY(dalloc(ctx, (void**)&L.tu, sizeof(float) * 2 * nn * wc));
  BIOT_TRY(dalloc(ctx, (void**)&L.tp, sizeof(float) * nn * wc));
  BIOT_TRY(dalloc(ctx, (void**)&L.val, sizeof(float) * ctx->nnz));
  BIOT_TRY(dalloc(ctx, (void**)&L.apval, sizeof(float) * ctx->n_pairs));
  if (ctx->prm.precision == BIOT_BF16VAL_FP32ACC) {
    BIOT_TRY(dalloc(ctx, (void**)&L.val_bf16, sizeof(__nv_bfloat16) * ctx->nnz));
    BIOT_TRY(dalloc(ctx, (void**)&L.apval_bf16, sizeof(__nv_bfloat16) * ctx->n_pairs));
  }
  return BIOT_OK;
}

void release_time_buffers(biot_ctx* ctx) {
  void** bufs[] = {(void**)&ctx->X,     (void**)&ctx->F,       (void**)&ctx->V,      (void**)&ctx->Z,
                   (void**)&ctx->Wv,    (void**)&ctx->part,    (void**)&ctx->colscal, (void**)&ctx->H,
                   (void**)&ctx->hvec,  (void**)&ctx->kcol,    (void**)&ctx->tu,     (void**)&ctx->tp,
                   (void**)&ctx->lp.V,   (void**)&ctx->lp.Z,
                   (void**)&ctx->lp.Wv, (void**)&ctx->lp.tu,   (void**)&ctx->lp.tp,  (void**)&ctx->lp.val,
                   (void**)&ctx->lp.apval, (void**)&ctx->lp.val_bf16, (void**)&ctx->lp.apval_bf16};
  for (void** b : bufs) {
    if (!*b) continue;
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), *b);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    cudaFree(*b);
    *b = nullptr;
  }
}

// Copy steps [lo, lo + nc) of a [dof][ld] device array to host[nc][n_dof] (staged through Wv).
biot_status copy_out_steps(biot_ctx* ctx, const double* src, int lds, int col0, int nc, const double* rowscale,
                           double* host) {
  const int nd = ctx->n_dof;
  for (int c = 0; c < nc; c += ctx->wcap) {
    const int m = std::min(ctx->wcap, nc - c);
    dim3 grid(div_up(nd, 32), div_up(m, 32)), block(32, 8);
    BIOT_LAUNCH(k_dof_to_step<double>, grid, block, 0, ctx->stream, src, lds, col0 + c, m, nd, rowscale, ctx->Wv);
    BIOT_CU(ctx, cudaGetLastError());
    BIOT_CU(ctx, cudaMemcpyAsync(host + (size_t)c * nd, ctx->Wv, sizeof(double) * nd * m, cudaMemcpyDeviceToHost,
                                 ctx->stream));
  }
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return BIOT_OK;
}

biot_status copy_in_steps(biot_ctx* ctx, const double* host, int nc, const double* rowscale, double* dst, int ldd,
                          int col0) {
  const int nd = ctx->n_dof;
  for (int c = 0; c < nc; c += ctx->wcap) {
    const int m = std::min(ctx->wcap, nc - c);
    BIOT_CU(ctx, cudaMemcpyAsync(ctx->Wv, host + (size_t)c * nd, sizeof(double) * nd * m, cudaMemcpyHostToDevice,
                                 ctx->stream));
    dim3 grid(div_up(nd, 32), div_up(m, 32)), block(32, 8);
    BIOT_LAUNCH(k_step_to_dof<double>, grid, block, 0, ctx->stream, ctx->Wv, m, nd, rowscale, dst, ldd, col0 + c);
    BIOT_CU(ctx, cudaGetLastError());
  }
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return BIOT_OK;
}

}  // namespace

biot_status fst_norm2_ctx(biot_ctx* ctx, double* out) { return fst_norm2(ctx, out); }
biot_status spacetime_residual_ctx(biot_ctx* ctx, double* out) { return spacetime_residual(ctx, out); }

}  // namespace biot

using namespace biot;

extern "C" {

biot_status biot_mesh_create(int32_t n, double Lx, double Ly, void* cuda_stream, biot_ctx** out) {
  if (!out) return fail(nullptr, BIOT_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 4096) return fail(nullptr, BIOT_E_INVALID, "n = %d outside 1..4096", n);
  if (!(Lx > 0.0) || !(Ly > 0.0)) return fail(nullptr, BIOT_E_INVALID, "domain size must be positive");
  biot_ctx* ctx = new (std::nothrow) biot_ctx();
  if (!ctx) return fail(nullptr, BIOT_E_OOM, "host allocation failed");
  ctx->n = n;
  ctx->Lx = Lx;
  ctx->Ly = Ly;
  ctx->stream = (cudaStream_t)cuda_stream;
  {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      biot_status st = fail(nullptr, BIOT_E_CUDA, "biot_mesh_create: side stream: %s", cudaGetErrorString(e));
      biot_destroy(ctx);
      return st;
    }
  }
  ctx->n_nodes = (n + 1) * (n + 1);
  ctx->n_dof = 3 * ctx->n_nodes;
  ctx->n_pairs = 7 * n * n + 6 * n + 1;
  ctx->nnz = 9LL * ctx->n_pairs;
  ctx->band_u = 2 * (n + 2) + 1;
  ctx->band_p = n + 2;
  biot_status st = BIOT_OK;
  do {
    if ((st = dalloc(ctx, (void**)&ctx->status, sizeof(int32_t))) != BIOT_OK) break;
    if ((st = dalloc(ctx, (void**)&ctx->val, sizeof(double) * ctx->nnz)) != BIOT_OK) break;
    if ((st = dalloc(ctx, (void**)&ctx->apval, sizeof(double) * ctx->n_pairs)) != BIOT_OK) break;
    if ((st = dalloc(ctx, (void**)&ctx->dsc, sizeof(double) * ctx->n_dof)) != BIOT_OK) break;
    if ((st = dalloc(ctx, (void**)&ctx->dsq, sizeof(double) * ctx->n_dof)) != BIOT_OK) break;
    if ((st = dalloc(ctx, (void**)&ctx->dmask, ctx->n_dof)) != BIOT_OK) break;
    if ((st = dalloc(ctx, (void**)&ctx->kappa, sizeof(double) * 2 * (size_t)n * n)) != BIOT_OK) break;
    if ((st = build_pattern(ctx)) != BIOT_OK) break;
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "pattern")) != BIOT_OK) break;
  } while (0);
  if (st != BIOT_OK) {
    g_create_error = ctx->err;
    dfree_all(ctx);
    delete ctx;
    return st;
  }
  *out = ctx;
  return BIOT_OK;
}

biot_status biot_assemble(biot_ctx* ctx, const biot_params* p) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  if (!p) return fail(ctx, BIOT_E_INVALID, "params is NULL");
  if (!(p->E > 0.0) || !(p->nu > -1.0 && p->nu < 0.5) || !(p->alpha > 0.0) || !(p->tau > 0.0))
    return fail(ctx, BIOT_E_INVALID, "material or time step out of range");
  if (p->n_t < 1 || p->n_iter < 1 || p->n_iter > kMaxIter)
    return fail(ctx, BIOT_E_INVALID, "n_t >= 1 and 1 <= n_iter <= %d required", kMaxIter);
  if (p->problem != BIOT_TERZAGHI && p->problem != BIOT_MMS_TRIG && p->problem != BIOT_BARRY_MERCER &&
      p->problem != BIOT_MANDEL)
    return fail(ctx, BIOT_E_INVALID, "problem");
  if (p->beta_mode < BIOT_BETA_H2 || p->beta_mode > BIOT_BETA_NONE) return fail(ctx, BIOT_E_INVALID, "beta_mode");
  if (p->schedule != BIOT_SCHED_TOL && p->schedule != BIOT_SCHED_PAPER && p->schedule != BIOT_SCHED_EAGER)
    return fail(ctx, BIOT_E_INVALID, "schedule");
  if (p->precision < BIOT_FP64 || p->precision > BIOT_BF16VAL_FP32ACC)
    return fail(ctx, BIOT_E_INVALID, "precision %d", p->precision);
  if (p->window < 0) return fail(ctx, BIOT_E_INVALID, "window must be >= 0");
  const size_t ne = 2 * (size_t)ctx->n * ctx->n;
  std::vector<double> kap(ne, p->kappa_const);
  if (p->kappa_elem) kap.assign(p->kappa_elem, p->kappa_elem + ne);
  for (double k : kap)
    if (!(k > 0.0) || !std::isfinite(k)) return fail(ctx, BIOT_E_INVALID, "permeability must be positive");
  const int wcap = std::max(1, std::min(p->n_t, p->window > 0 ? p->window : p->n_t));
  if (ctx->X && (p->n_t != ctx->n_t || wcap != ctx->wcap || p->n_iter != ctx->n_iter ||
                 p->precision != ctx->prm.precision)) {
    release_time_buffers(ctx);
    ctx->assembled = false;
  }
  ctx->prm = *p;
  ctx->prm.kappa_elem = nullptr;
  ctx->precond = 0;
  if (!ctx->X) {
    ctx->n_t = p->n_t;
    ctx->ldx = p->n_t + 1;
    ctx->wcap = wcap;
    ctx->n_iter = p->n_iter;
    BIOT_TRY(alloc_time_buffers(ctx));
  }
  BIOT_CU(ctx, cudaMemcpyAsync(ctx->kappa, kap.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, ctx->stream));
  BIOT_TRY(assemble_system(ctx));
  if (low_precision(ctx)) {
    BIOT_LAUNCH(k_cvt_f32, 1024, 256, 0, ctx->stream, ctx->val, ctx->lp.val, (size_t)ctx->nnz);
    BIOT_LAUNCH(k_cvt_f32, 256, 256, 0, ctx->stream, ctx->apval, ctx->lp.apval, (size_t)ctx->n_pairs);
    if (ctx->prm.precision == BIOT_BF16VAL_FP32ACC) {
      BIOT_LAUNCH(k_cvt_bf16, 1024, 256, 0, ctx->stream, ctx->val, ctx->lp.val_bf16, (size_t)ctx->nnz);
      BIOT_LAUNCH(k_cvt_bf16, 256, 256, 0, ctx->stream, ctx->apval, ctx->lp.apval_bf16, (size_t)ctx->n_pairs);
    }
    BIOT_CU(ctx, cudaGetLastError());
  }
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->assembled = true;
  return BIOT_OK;
}

biot_status biot_precond_setup(biot_ctx* ctx, int32_t kind) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  if (kind != BIOT_PRECOND_TRI && kind != BIOT_PRECOND_DIAG) return fail(ctx, BIOT_E_INVALID, "precond kind %d", kind);
  ctx->precond = 0;
  if (ctx->inner == BIOT_INNER_GMG) {
    BIOT_TRY(gmg_setup(ctx));
    ctx->precond = kind;
  } else {
    gmg_free(ctx);
    BIOT_TRY(band_setup(ctx, kind));
  }
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return BIOT_OK;
}

biot_status biot_set_inner_solver(biot_ctx* ctx, int32_t kind, int32_t levels, int32_t cycles, int32_t smooth) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  if (kind != BIOT_INNER_EXACT && kind != BIOT_INNER_GMG) return fail(ctx, BIOT_E_INVALID, "inner solver %d", kind);
  if (kind == BIOT_INNER_GMG) {
    if (levels < 0 || levels == 1 || cycles < 1 || cycles > 16 || smooth < 1 || smooth > 8)
      return fail(ctx, BIOT_E_INVALID, "multigrid: levels 0 or >= 2, cycles 1..16, smoothing steps 1..8");
    if (gmg_levels_for(ctx->n, levels) < 2)
      return fail(ctx, BIOT_E_INVALID, "multigrid: n = %d cannot be coarsened (%s)", ctx->n,
                  levels == 0 ? "automatic depth needs an even n above 16" : "n odd or below 4");
    ctx->gmg_levels_req = levels;
    ctx->gmg_cycles = cycles;
    ctx->gmg_smooth = smooth;
  }
  ctx->inner = kind;
  return BIOT_OK;
}

biot_status biot_set_substructure(biot_ctx* ctx, int32_t strips) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  if (strips < 0 || (strips >= 2 && 3 * strips > ctx->n + 2))
    return fail(ctx, BIOT_E_INVALID, "strips = %d: need 0, 1 or 2 .. (n + 2) / 3 at n = %d", strips, ctx->n);
  ctx->sub_req = strips;
  return BIOT_OK;
}

biot_status biot_sweep(biot_ctx* ctx, int32_t lo, int32_t hi, double* rel_out) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_precond(ctx));
  BIOT_TRY(check_window(ctx, lo, hi));
  BIOT_TRY(sweep_impl(ctx, lo, hi, rel_out));
  if (!rel_out) BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

biot_status biot_residual_norms(biot_ctx* ctx, int32_t lo, int32_t hi, double* rel_out) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  BIOT_TRY(check_window(ctx, lo, hi));
  if (!rel_out) return fail(ctx, BIOT_E_INVALID, "rel_out is NULL");
  return residual_window(ctx, lo, hi - lo + 1, rel_out);
}

biot_status biot_set_schedule(biot_ctx* ctx, int32_t schedule) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  if (schedule != BIOT_SCHED_TOL && schedule != BIOT_SCHED_PAPER && schedule != BIOT_SCHED_EAGER)
    return fail(ctx, BIOT_E_INVALID, "schedule %d", schedule);
  if (schedule == BIOT_SCHED_PAPER && ctx->prm.window > ctx->wcap)
    return fail(ctx, BIOT_E_INVALID, "paper schedule needs window <= %d", ctx->wcap);
  ctx->prm.schedule = schedule;
  return BIOT_OK;
}

biot_status biot_pint_solve(biot_ctx* ctx, double tol, int32_t max_outer, int32_t* sweeps_done,
                            double* final_rel_res) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_precond(ctx));
  if (max_outer < 1) return fail(ctx, BIOT_E_INVALID, "max_outer must be >= 1");
  if (ctx->prm.schedule != BIOT_SCHED_PAPER && !(tol >= 0.0))
    return fail(ctx, BIOT_E_INVALID, "tol must be >= 0");
  const int n_t = ctx->n_t;
  int w = 0;
  biot_status result = BIOT_OK;
  // every solve starts with a clear device status (a timed-out wait of an earlier call
  // does not carry over)
  BIOT_CU(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
  if (ctx->prm.schedule == BIOT_SCHED_PAPER) {
    const int M = ctx->prm.window > 0 ? ctx->prm.window : n_t;
    if (M > ctx->wcap) return fail(ctx, BIOT_E_INVALID, "paper schedule needs window <= %d", ctx->wcap);
    const int total = n_t + M - 1;
    for (w = 1; w <= total; ++w) {
      if (w > max_outer) {
        --w;
        result = fail(ctx, BIOT_E_NOT_CONVERGED, "paper schedule stopped after %d of %d sweeps", max_outer, total);
        break;
      }
      const int a = std::max(1, w - M + 1), z = std::min(w, n_t);
      BIOT_TRY(sweep_impl(ctx, a, z, nullptr));
    }
    if (result == BIOT_OK) w = total;
  } else {
    bool conv = false;
    if (low_precision(ctx)) BIOT_TRY(tol_schedule<float>(ctx, tol, max_outer, 0, &w, &conv));
    else BIOT_TRY(tol_schedule<double>(ctx, tol, max_outer, 0, &w, &conv));
    if (!conv) result = fail(ctx, BIOT_E_NOT_CONVERGED, "tolerance %.3g not met after %d sweeps", tol, max_outer);
  }
  if (sweeps_done) *sweeps_done = w;
  if (final_rel_res) BIOT_TRY(spacetime_residual(ctx, final_rel_res));
  BIOT_TRY(device_status(ctx));
  return result;
}

biot_status biot_get_solution(const biot_ctx* cctx, int32_t step, double* host_out) {
  biot_ctx* ctx = const_cast<biot_ctx*>(cctx);
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  if (!host_out || step < 0 || step > ctx->n_t) return fail(ctx, BIOT_E_INVALID, "step %d outside 0..%d", step, ctx->n_t);
  return copy_out_steps(ctx, ctx->X, ctx->ldx, step, 1, nullptr, host_out);
}

biot_status biot_get_state(const biot_ctx* cctx, int32_t lo, int32_t hi, double* host) {
  biot_ctx* ctx = const_cast<biot_ctx*>(cctx);
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  if (!host || lo < 0 || hi > ctx->n_t || lo > hi) return fail(ctx, BIOT_E_INVALID, "bad state range");
  return copy_out_steps(ctx, ctx->X, ctx->ldx, lo, hi - lo + 1, nullptr, host);
}

biot_status biot_set_state(biot_ctx* ctx, int32_t lo, int32_t hi, const double* host) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  if (!host || lo < 0 || hi > ctx->n_t || lo > hi) return fail(ctx, BIOT_E_INVALID, "bad state range");
  return copy_in_steps(ctx, host, hi - lo + 1, nullptr, ctx->X, ctx->ldx, lo);
}

biot_status biot_get_csr(const biot_ctx* cctx, int32_t* rowptr, int32_t* col, double* val, double* ap_pp,
                         int64_t* nnz_out) {
  biot_ctx* ctx = const_cast<biot_ctx*>(cctx);
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  if (nnz_out) *nnz_out = ctx->nnz;
  cudaStream_t s = ctx->stream;
  if (rowptr)
    BIOT_CU(ctx, cudaMemcpyAsync(rowptr, ctx->rowptr, sizeof(int32_t) * (ctx->n_dof + 1), cudaMemcpyDeviceToHost, s));
  if (col) BIOT_CU(ctx, cudaMemcpyAsync(col, ctx->col, sizeof(int32_t) * ctx->nnz, cudaMemcpyDeviceToHost, s));
  if (val || ap_pp) BIOT_TRY(need_assembled(ctx));
  if (val) BIOT_CU(ctx, cudaMemcpyAsync(val, ctx->val, sizeof(double) * ctx->nnz, cudaMemcpyDeviceToHost, s));
  if (ap_pp) BIOT_CU(ctx, cudaMemcpyAsync(ap_pp, ctx->apval, sizeof(double) * ctx->n_pairs, cudaMemcpyDeviceToHost, s));
  BIOT_CU(ctx, cudaStreamSynchronize(s));
  return BIOT_OK;
}

biot_status biot_get_rhs(const biot_ctx* cctx, double* host) {
  biot_ctx* ctx = const_cast<biot_ctx*>(cctx);
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  if (!host) return fail(ctx, BIOT_E_INVALID, "host is NULL");
  return copy_out_steps(ctx, ctx->F, ctx->ldx, 0, ctx->n_t + 1, nullptr, host);
}

biot_status biot_get_residual(biot_ctx* ctx, int32_t lo, int32_t hi, double* host) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_assembled(ctx));
  BIOT_TRY(check_window(ctx, lo, hi));
  if (!host) return fail(ctx, BIOT_E_INVALID, "host is NULL");
  BIOT_TRY(residual_window(ctx, lo, hi - lo + 1, nullptr));
  // V_0 holds d .* r; undo the equilibration while transposing.
  return copy_out_steps(ctx, ctx->V, ctx->wcap, 0, hi - lo + 1, ctx->dsc, host);
}

biot_status biot_precond_apply(biot_ctx* ctx, int32_t ncols, const double* host_in, double* host_out) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_precond(ctx));
  if (ncols < 1 || ncols > ctx->wcap || !host_in || !host_out)
    return fail(ctx, BIOT_E_INVALID, "ncols must be in 1..%d and buffers non-NULL", ctx->wcap);
  // precond_apply computes P^{-1}(V ./ d); load V = d .* in.
  if (!low_precision(ctx)) {
    BIOT_TRY(copy_in_steps(ctx, host_in, ncols, ctx->dsc, ctx->V, ctx->wcap, 0));
    precond_apply<double>(ctx, ctx->V, ctx->Z, 0, ncols);
    BIOT_CU(ctx, cudaGetLastError());
    return copy_out_steps(ctx, ctx->Z, ctx->wcap, 0, ncols, nullptr, host_out);
  }
  // reduced precision: the FP32 preconditioner of the correction sweep
  const int nd = ctx->n_dof;
  dim3 grid(div_up(nd, 32), div_up(ncols, 32)), block(32, 8);
  BIOT_CU(ctx, cudaMemcpyAsync(ctx->Wv, host_in, sizeof(double) * nd * ncols, cudaMemcpyHostToDevice, ctx->stream));
  BIOT_LAUNCH(k_step_to_dof<float>, grid, block, 0, ctx->stream, ctx->Wv, ncols, nd, ctx->dsc, ctx->lp.V, ctx->wcap,
              0);
  precond_apply<float>(ctx, ctx->lp.V, ctx->lp.Z, 0, ncols);
  BIOT_LAUNCH(k_dof_to_step<float>, grid, block, 0, ctx->stream, ctx->lp.Z, ctx->wcap, 0, ncols, nd, nullptr, ctx->Wv);
  BIOT_CU(ctx, cudaGetLastError());
  BIOT_CU(ctx, cudaMemcpyAsync(host_out, ctx->Wv, sizeof(double) * nd * ncols, cudaMemcpyDeviceToHost, ctx->stream));
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return BIOT_OK;
}

biot_status biot_get_info(const biot_ctx* ctx, biot_info* out) {
  if (bad_ctx(ctx) || !out) return fail(nullptr, BIOT_E_INVALID, "NULL argument");
  out->n = ctx->n;
  out->n_nodes = ctx->n_nodes;
  out->n_dof = ctx->n_dof;
  out->nnz = ctx->nnz;
  out->n_pairs = ctx->n_pairs;
  out->n_t = ctx->n_t;
  out->window_cap = ctx->wcap;
  out->band_u = ctx->band_u;
  out->band_p = ctx->band_p;
  out->precond = ctx->precond;
  out->precision = ctx->prm.precision;
  out->beta = ctx->beta;
  out->device_bytes = ctx->device_bytes;
  out->inner = ctx->inner;
  gmg_info(ctx, &out->gmg_levels, &out->gmg_lam_u, &out->gmg_lam_p);
  return BIOT_OK;
}

biot_status biot_timing_enable(biot_ctx* ctx, int32_t enable) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->timing = enable != 0;
  ctx->ev_used = 0;
  for (auto& m : ctx->ev_marks) m.clear();
  return BIOT_OK;
}

biot_status biot_timing_read(biot_ctx* ctx, int32_t kc, double* total_ms, int64_t* launches) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  if (kc < 0 || kc >= BIOT_KC_COUNT || !total_ms || !launches) return fail(ctx, BIOT_E_INVALID, "kernel class");
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  double sum = 0.0;
  for (auto& pr : ctx->ev_marks[kc]) {
    float ms = 0.f;
    BIOT_CU(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[pr.first], ctx->ev_pool[pr.second]));
    sum += ms;
  }
  *total_ms = sum;
  *launches = (int64_t)ctx->ev_marks[kc].size();
  return BIOT_OK;
}

biot_status biot_tune(biot_ctx* ctx, const char* cache_path, biot_tuning* out) {
  if (bad_ctx(ctx)) return fail(nullptr, BIOT_E_INVALID, "ctx is NULL");
  BIOT_TRY(need_precond(ctx));
  // the SpMM shape (reduced-precision sweeps), for every kind of block solve
  std::map<std::string, int> cache = read_tune_cache(cache_path);
  int sp_hit = 0;
  double sp_ms = 0.0, sp_def = 0.0;
  BIOT_TRY(spmm_tune(ctx, &cache, &sp_hit, &sp_ms, &sp_def));
  const bool sp_cached = sp_hit || !low_precision(ctx);
  auto finish = [&](biot_tuning res, bool hits) -> biot_status {
    res.spmm_variant = ctx->spmm_var;
    res.ms_spmm = sp_ms;
    res.ms_spmm_default = sp_def;
    res.from_cache = (hits && sp_cached) ? 1 : 0;
    if (!res.from_cache) write_tune_cache(cache_path, cache);
    if (out) *out = res;
    return BIOT_OK;
  };
  if (ctx->gmg) return finish(biot_tuning{}, true);  // multigrid block solves: no band-solve variants
  const bool fp64 = !low_precision(ctx);
  const int pi = fp64 ? 0 : 1;
  const int nc = ctx->wcap;
  const int bu = ctx->band_u, bp = ctx->band_p;
  const std::string ku = tune_key(fp64, 2 * ctx->n_nodes, bu, nc), kp = tune_key(fp64, ctx->n_nodes, bp, nc);
  biot_tuning res{};
  res.from_cache = 0;
  if (ctx->sub[0]) {
    // substructured block solves: time the interior and separator variants of A and S (or
    // take them from the cache, keyed "sub:" + precision, rows, half-band and window)
    double ms[2] = {0.0, 0.0}, ms_sep[2] = {0.0, 0.0};
    int hits = 0;
    BIOT_TRY(sub_tune(ctx, ms, ms_sep, &cache, &hits));
    BIOT_TRY(device_status(ctx));
    const SubBlock* su = ctx->sub[0];
    const SubBlock* sp = ctx->sub[1];
    res.ms_u = ms[0];
    res.ms_p = ms[1];
    res.variant_u = su->varI[pi];
    res.variant_p = sp->varI[pi];
    res.tma_u = kBandVariants[res.variant_u].tma;
    res.nb_u = kBandVariants[res.variant_u].nb;
    res.threads_u = kBandVariants[res.variant_u].threads;
    res.tma_p = kBandVariants[res.variant_p].tma;
    res.nb_p = kBandVariants[res.variant_p].nb;
    res.threads_p = kBandVariants[res.variant_p].threads;
    res.strips = su->k;
    res.variant_sep_u = su->varS[pi];
    res.variant_sep_p = sp->varS[pi];
    res.ms_sep_u = ms_sep[0];
    res.ms_sep_p = ms_sep[1];
    return finish(res, hits == 4);
  }
  const int def_u = band_variant_default(fp64, bu), def_p = band_variant_default(fp64, bp);
  // clean inputs for the timing runs
  const size_t es = fp64 ? 8 : 4;
  void* vin = fp64 ? (void*)ctx->V : (void*)ctx->lp.V;
  void* z = fp64 ? (void*)ctx->Z : (void*)ctx->lp.Z;
  BIOT_CU(ctx, cudaMemsetAsync(vin, 0, es * (size_t)ctx->n_dof * nc, ctx->stream));
  auto time_pair = [&](bool u, int v) -> float {
    return fp64 ? time_band_pair<double>(ctx, u, v, (const double*)vin, (double*)z, nc)
                : time_band_pair<float>(ctx, u, v, (const float*)vin, (float*)z, nc);
  };
  bool hit_u = cache.count(ku) && band_variant_ok(cache[ku], fp64, bu);
  bool hit_p = cache.count(kp) && band_variant_ok(cache[kp], fp64, bp);
  for (int which = 0; which < 2; ++which) {
    const bool u = which == 0;
    const int b = u ? bu : bp;
    int best = u ? def_u : def_p;
    float tbest = time_pair(u, best);
    (u ? res.ms_u_default : res.ms_p_default) = tbest;
    if (u ? hit_u : hit_p) {
      best = cache[u ? ku : kp];
      tbest = time_pair(u, best);
    } else {
      for (int v = 0; v < kBandVariantCount; ++v) {
        if (!band_variant_ok(v, fp64, b) || v == (u ? def_u : def_p)) continue;
        const float t = time_pair(u, v);
        if (t < tbest) {
          tbest = t;
          best = v;
        }
      }
      cache[u ? ku : kp] = best;
    }
    BIOT_CU(ctx, cudaGetLastError());
    BIOT_TRY(ensure_dnb(ctx, fp64, u, best));
    if (u) {
      ctx->band_var_u[pi] = best;
      res.variant_u = best;
      res.ms_u = tbest;
    } else {
      ctx->band_var_p[pi] = best;
      res.variant_p = best;
      res.ms_p = tbest;
    }
  }
  BIOT_TRY(device_status(ctx));
  res.tma_u = kBandVariants[res.variant_u].tma;
  res.nb_u = kBandVariants[res.variant_u].nb;
  res.threads_u = kBandVariants[res.variant_u].threads;
  res.tma_p = kBandVariants[res.variant_p].tma;
  res.nb_p = kBandVariants[res.variant_p].nb;
  res.threads_p = kBandVariants[res.variant_p].threads;
  return finish(res, hit_u && hit_p);
}

int64_t biot_launch_count(void) { return g_launches.load(); }

const char* biot_last_error(const biot_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.empty() ? "no error" : ctx->err.c_str();
}

void biot_destroy(biot_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  gmg_free(ctx);  // destroys the multigrid level contexts
  sub_free(ctx);  // synchronises both streams: before the side stream is destroyed
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
    ctx->side = nullptr;
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  ctx->ev_fork = ctx->ev_join = nullptr;
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  dfree_all(ctx);
  delete ctx;
}

}  // extern "C"
