// Exact block solves of the preconditioners P1 (Eq. p1) and P2 (Eq. p2).
//
// Both preconditioners need A^{-1} (elasticity block) and S^{-1}, S = (tau +
// beta/K) C = tau C + beta L (approximate Schur complement, Sec. 3.1). On the
// structured grid both are banded: with the u-ordering 2 v + f the half-band
// of A is 2 (n + 2) + 1, and S in node order has half-band n + 2. Both are SPD
// after the symmetric Dirichlet elimination, so they are factored once by band
// Cholesky (A = L L^T) on the device, and every preconditioner application is
// two band triangular solves per block: exact up to rounding, as the paper's
// P^{-1} requires.
//
// Storage: lower band rows, Lb[i][q] = L[i][i - b + q], q = 0..b (diagonal at q = b);
// the transposed band Ub[i][q] = L[i + q][i] (diagonal at q = 0) serves the
// backward solve with contiguous rows.
//
// The triangular solves run one CTA per active time step (column); the last b
// solution values live in a shared-memory ring, the band row of the next row is
// prefetched into registers while the current row is reduced.
#include "common.cuh"

namespace biot {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kMaxQ = 9;          // band rows up to kMaxQ * 256 entries (n <= 1147)
constexpr int kRing = 4096;       // power of two >= b + 1
constexpr int kRhsChunk = 256;

__global__ void k_band_extract_u(int nn, int bu, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ Lb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // u-row 2 v + f
  if (i >= 2 * nn) return;
  const int r = 3 * (i >> 1) + (i & 1);
  for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
    const int c = col[e];
    const int g = c % 3;
    if (g == 2) continue;
    const int j = 2 * (c / 3) + g;
    if (j > i || i - j > bu) continue;
    Lb[(size_t)i * (bu + 1) + (bu - (i - j))] = val[e];
  }
}

__global__ void k_band_extract_p(int nn, int bp, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ Lb) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nn) return;
  const int r = 3 * v + 2;
  for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
    const int c = col[e];
    if (c % 3 != 2) continue;
    const int j = c / 3;
    if (j > v || v - j > bp) continue;
    Lb[(size_t)v * (bp + 1) + (bp - (v - j))] = -val[e];  // S = -AA_pp
  }
}

// Column j of the right-looking band Cholesky: L_jj = sqrt(a_jj), L_ij = a_ij / L_jj.
__global__ void k_chol_scale(int N, int b, int j, double* __restrict__ Lb, int32_t* __restrict__ status) {
  if (*status != 0) return;
  const double d = Lb[(size_t)j * (b + 1) + b];
  if (!(d > 0.0)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *status = j + 1;
    return;
  }
  const double s = sqrt(d);
  const double inv = 1.0 / s;
  const int last = min(N - 1, j + b);
  for (int i = j + 1 + blockIdx.x * blockDim.x + threadIdx.x; i <= last; i += blockDim.x * gridDim.x)
    Lb[(size_t)i * (b + 1) + (b - (i - j))] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) Lb[(size_t)j * (b + 1) + b] = s;
}

// Trailing update a_ik -= L_ij L_kj for j < k <= i <= j + b.
__global__ void k_chol_update(int N, int b, int j, double* __restrict__ Lb, const int32_t* __restrict__ status) {
  if (*status != 0) return;
  const int last = min(N - 1, j + b);
  const int m = last - j;  // rows j+1..last
  const long long tri = (long long)m * (m + 1) / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tri; t += (long long)blockDim.x * gridDim.x) {
    // t -> (ii, kk), 0 <= kk <= ii < m
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)ii * (ii + 1) / 2 > t) --ii;
    while ((long long)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    const int kk = (int)(t - (long long)ii * (ii + 1) / 2);
    const int i = j + 1 + ii, k = j + 1 + kk;
    const double lij = Lb[(size_t)i * (b + 1) + (b - (i - j))];
    const double lkj = Lb[(size_t)k * (b + 1) + (b - (k - j))];
    Lb[(size_t)i * (b + 1) + (b - (i - k))] -= lij * lkj;
  }
}

__global__ void k_band_transpose(int N, int b, const double* __restrict__ Lb, double* __restrict__ Ub) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)N * (b + 1)) return;
  const int i = (int)(t / (b + 1)), q = (int)(t % (b + 1));
  Ub[t] = (i + q < N) ? Lb[(size_t)(i + q) * (b + 1) + (b - q)] : 0.0;
}

enum SolveMode {
  FWD_U_FROM_V = 0,   // rhs_i = vin[u-dof(i)] / d,     out ty[i]
  FWD_P_FROM_T = 1,   // rhs_i = tp[i],                 out tp[i]
  FWD_P_FROM_V = 2,   // rhs_i = -vin[3i+2] / d,        out tp[i]
  BWD_U_TO_Z = 3,     // rhs_i = ty[i],                 out z[u-dof(i)]
  BWD_P_TO_Z = 4      // rhs_i = tp[i],                 out z[3i+2]
};

__device__ __forceinline__ int udof(int i) { return 3 * (i >> 1) + (i & 1); }

// One band triangular solve per CTA (column c = c0 + blockIdx.x).
// Forward: y_i = (rhs_i - sum_{q<b} Lb[i][q] y_{i-b+q}) / Lb[i][b], i ascending.
// Backward: x_i = (rhs_i - sum_{q>=1} Ub[i][q] x_{i+q}) / Ub[i][0], i descending.
template <int MODE>
__global__ void __launch_bounds__(kSolveThreads)
k_band_solve(int N, int b, const double* __restrict__ band, const double* __restrict__ vin,
             const double* __restrict__ dsc, double* __restrict__ ty, double* __restrict__ tp,
             double* __restrict__ z, int ld, int c0) {
  constexpr bool kFwd = MODE <= FWD_P_FROM_V;
  __shared__ double ring[kRing];
  __shared__ double rhs[kRhsChunk];
  __shared__ double red[kSolveThreads / 32];
  __shared__ double sdiag;
  const int c = c0 + blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int W = b + 1;
  // register prefetch of the band row for the next step
  double lnext[kMaxQ];
  auto row_of = [&](int step) { return kFwd ? step : (N - 1 - step); };
  auto load_row = [&](int step, double* dst) {
    const int i = row_of(step);
    const double* rowp = band + (size_t)i * W;
#pragma unroll
    for (int u = 0; u < kMaxQ; ++u) {
      const int q = t + u * kSolveThreads;
      dst[u] = (q < W) ? rowp[q] : 0.0;
    }
  };
  auto read_rhs = [&](int i) -> double {
    if (MODE == FWD_U_FROM_V) { const int r = udof(i); return vin[(size_t)r * ld + c] / dsc[r]; }
    if (MODE == FWD_P_FROM_T) return tp[(size_t)i * ld + c];
    if (MODE == FWD_P_FROM_V) { const int r = 3 * i + 2; return -vin[(size_t)r * ld + c] / dsc[r]; }
    if (MODE == BWD_U_TO_Z) return ty[(size_t)i * ld + c];
    return tp[(size_t)i * ld + c];
  };
  auto write_out = [&](int i, double y) {
    if (MODE == FWD_U_FROM_V) ty[(size_t)i * ld + c] = y;
    else if (MODE == FWD_P_FROM_T || MODE == FWD_P_FROM_V) tp[(size_t)i * ld + c] = y;
    else if (MODE == BWD_U_TO_Z) z[(size_t)udof(i) * ld + c] = y;
    else z[(size_t)(3 * i + 2) * ld + c] = y;
  };
  if (N > 0) load_row(0, lnext);
  for (int step = 0; step < N; ++step) {
    const int i = row_of(step);
    if ((step % kRhsChunk) == 0) {
      __syncthreads();
      for (int u = t; u < kRhsChunk; u += kSolveThreads) {
        const int s2 = step + u;
        rhs[u] = (s2 < N) ? read_rhs(row_of(s2)) : 0.0;
      }
      __syncthreads();
    }
    double lcur[kMaxQ];
#pragma unroll
    for (int u = 0; u < kMaxQ; ++u) lcur[u] = lnext[u];
    if (step + 1 < N) load_row(step + 1, lnext);
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kMaxQ; ++u) {
      const int q = t + u * kSolveThreads;
      if (kFwd) {
        // entries q < b couple row i to row i - b + q (must exist: i - b + q >= 0)
        if (q < b && i - b + q >= 0) s += lcur[u] * ring[(i - b + q) & (kRing - 1)];
      } else {
        if (q >= 1 && q <= b && i + q < N) s += lcur[u] * ring[(i + q) & (kRing - 1)];
      }
    }
#pragma unroll
    for (int u = 0; u < kMaxQ; ++u)
      if (t + u * kSolveThreads == (kFwd ? b : 0)) sdiag = lcur[u];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < kSolveThreads / 32; ++w) tot += red[w];
      const double y = (rhs[step % kRhsChunk] - tot) / sdiag;
      ring[i & (kRing - 1)] = y;
      write_out(i, y);
    }
    __syncthreads();
  }
}

// Full band Cholesky of an SPD band matrix held in Lb (in place).
biot_status band_cholesky(biot_ctx* ctx, int N, int b, double* Lb) {
  BIOT_CU(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
  const long long tri = (long long)b * (b + 1) / 2;
  const int ublocks = (int)((tri + 255) / 256 < 1024 ? (tri + 255) / 256 : 1024);
  for (int j = 0; j < N; ++j) {
    BIOT_LAUNCH(k_chol_scale, 1, 256, 0, ctx->stream, N, b, j, Lb, ctx->status);
    if (j + 1 < N) BIOT_LAUNCH(k_chol_update, ublocks, 256, 0, ctx->stream, N, b, j, Lb, ctx->status);
  }
  BIOT_CU(ctx, cudaGetLastError());
  int32_t st = 0;
  BIOT_CU(ctx, cudaMemcpyAsync(&st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  if (st != 0) return fail(ctx, BIOT_E_CUDA, "band Cholesky: non-positive pivot at row %d", st - 1);
  return BIOT_OK;
}

}  // namespace

biot_status band_setup(biot_ctx* ctx, int kind) {
  const int nn = ctx->n_nodes;
  const int bu = ctx->band_u, bp = ctx->band_p;
  if (bu + 1 > kMaxQ * kSolveThreads || bu + 1 > kRing)
    return fail(ctx, BIOT_E_INVALID, "mesh too large for the band solver (half-band %d)", bu);
  const size_t su = (size_t)2 * nn * (bu + 1), sp = (size_t)nn * (bp + 1);
  if (!ctx->Lu) {
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Lu, sizeof(double) * su));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Uu, sizeof(double) * su));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Lp, sizeof(double) * sp));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Up, sizeof(double) * sp));
  }
  cudaStream_t s = ctx->stream;
  BIOT_CU(ctx, cudaMemsetAsync(ctx->Lu, 0, sizeof(double) * su, s));
  BIOT_CU(ctx, cudaMemsetAsync(ctx->Lp, 0, sizeof(double) * sp, s));
  BIOT_LAUNCH(k_band_extract_u, div_up(2 * nn, 256), 256, 0, s, nn, bu, ctx->rowptr, ctx->col, ctx->val, ctx->Lu);
  BIOT_LAUNCH(k_band_extract_p, div_up(nn, 256), 256, 0, s, nn, bp, ctx->rowptr, ctx->col, ctx->val, ctx->Lp);
  BIOT_TRY(band_cholesky(ctx, 2 * nn, bu, ctx->Lu));
  BIOT_TRY(band_cholesky(ctx, nn, bp, ctx->Lp));
  BIOT_LAUNCH(k_band_transpose, div_up((long long)su, 256), 256, 0, s, 2 * nn, bu, ctx->Lu, ctx->Uu);
  BIOT_LAUNCH(k_band_transpose, div_up((long long)sp, 256), 256, 0, s, nn, bp, ctx->Lp, ctx->Up);
  BIOT_CU(ctx, cudaGetLastError());
  ctx->precond = kind;
  return BIOT_OK;
}

void precond_apply(biot_ctx* ctx, const double* vin, double* z, int c0, int ncols) {
  const int nn = ctx->n_nodes, ld = ctx->wcap;
  cudaStream_t s = ctx->stream;
  BIOT_LAUNCH(k_band_solve<FWD_U_FROM_V>, ncols, kSolveThreads, 0, s, 2 * nn, ctx->band_u, ctx->Lu, vin, ctx->dsc,
              ctx->tu, ctx->tp, z, ld, c0);
  BIOT_LAUNCH(k_band_solve<BWD_U_TO_Z>, ncols, kSolveThreads, 0, s, 2 * nn, ctx->band_u, ctx->Uu, vin, ctx->dsc,
              ctx->tu, ctx->tp, z, ld, c0);
  if (ctx->precond == BIOT_PRECOND_TRI) {
    launch_coupling(ctx, z, vin, ctx->tp, c0, ncols);
    BIOT_LAUNCH(k_band_solve<FWD_P_FROM_T>, ncols, kSolveThreads, 0, s, nn, ctx->band_p, ctx->Lp, vin, ctx->dsc,
                ctx->tu, ctx->tp, z, ld, c0);
  } else {
    BIOT_LAUNCH(k_band_solve<FWD_P_FROM_V>, ncols, kSolveThreads, 0, s, nn, ctx->band_p, ctx->Lp, vin, ctx->dsc,
                ctx->tu, ctx->tp, z, ld, c0);
  }
  BIOT_LAUNCH(k_band_solve<BWD_P_TO_Z>, ncols, kSolveThreads, 0, s, nn, ctx->band_p, ctx->Up, vin, ctx->dsc, ctx->tu,
              ctx->tp, z, ld, c0);
}

}  // namespace biot
