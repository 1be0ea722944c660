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
// The triangular solves are blocked by kNB rows. For a block of rows, the part of
// each row's band that reaches into earlier blocks is a dense product with the
// solution history (every FMA useful, K-split over 4 lanes); the part inside the
// block is applied as the precomputed inverse of the block's triangle (a small
// dense product instead of a serial substitution). A CTA owns kCols time steps
// (columns); the last b + kNB solution rows live in a shared-memory ring. FP64
// throughput on GB300 is 2 FMA/clk/SM, so the design spends FP64 issue slots only
// on the band products: no per-row reduction trees, no divisions.
#include "common.cuh"

#include <algorithm>
#include <type_traits>

namespace biot {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kKSplit = kSolveThreads / kNB;    // lanes sharing one row's band product
constexpr int kCols = 2;                        // time steps (columns) per CTA


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
    Lb[(size_t)i * band_ld(bu) + (bu - (i - j))] = val[e];
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
    Lb[(size_t)v * band_ld(bp) + (bp - (v - j))] = -val[e];  // S = -AA_pp
  }
}

// Blocked right-looking band Cholesky, panels of kPanel columns.
// Panel kernel (one CTA): factors columns j0 .. j0 + np - 1 including the rows
// below them inside the band: L_jj = sqrt(a_jj), L_ij = a_ij / L_jj, and the
// rank-1 updates of the remaining panel columns.
constexpr int kPanel = 32;

__global__ void __launch_bounds__(256)
k_chol_panel(int N, int b, int j0, int np, double* __restrict__ Lb, int32_t* __restrict__ status) {
  __shared__ double sd;
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = (*status != 0);
  __syncthreads();
  if (bad) return;
  const size_t W = (size_t)band_ld(b);
  for (int jj = 0; jj < np; ++jj) {
    const int j = j0 + jj;
    if (t == 0) {
      const double d = Lb[(size_t)j * W + b];
      if (!(d > 0.0)) {
        *status = j + 1;
        bad = 1;
      } else {
        sd = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) return;
    const int last = min(N - 1, j + b);
    const double inv = 1.0 / sd;
    for (int i = j + 1 + t; i <= last; i += blockDim.x) Lb[(size_t)i * W + (b - (i - j))] *= inv;
    if (t == 0) Lb[(size_t)j * W + b] = sd;
    __syncthreads();
    for (int k = j + 1; k < j0 + np; ++k) {
      const double lkj = Lb[(size_t)k * W + (b - (k - j))];
      for (int i = k + t; i <= last; i += blockDim.x)
        Lb[(size_t)i * W + (b - (i - k))] -= Lb[(size_t)i * W + (b - (i - j))] * lkj;
    }
    __syncthreads();
  }
}

// Trailing update after a panel: a_ik -= sum_{j in panel} L_ij L_kj for
// j1 <= k <= i <= min(N - 1, j1 - 1 + b), j1 = j0 + np.
__global__ void k_chol_trailing(int N, int b, int j0, int np, double* __restrict__ Lb,
                                const int32_t* __restrict__ status) {
  if (*status != 0) return;
  const int j1 = j0 + np;
  const int last = min(N - 1, j1 - 1 + b);
  const int m = last - j1 + 1;
  if (m <= 0) return;
  const size_t W = (size_t)band_ld(b);
  const long long tri = (long long)m * (m + 1) / 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tri; t += (long long)blockDim.x * gridDim.x) {
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)ii * (ii + 1) / 2 > t) --ii;
    while ((long long)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    const int kk = (int)(t - (long long)ii * (ii + 1) / 2);
    const int i = j1 + ii, k = j1 + kk;
    const int jb = max(j0, i - b);
    double acc = 0.0;
    for (int j = jb; j < j1; ++j) acc += Lb[(size_t)i * W + (b - (i - j))] * Lb[(size_t)k * W + (b - (k - j))];
    Lb[(size_t)i * W + (b - (i - k))] -= acc;
  }
}

__global__ void k_band_transpose(int N, int b, const double* __restrict__ Lb, double* __restrict__ Ub) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)N * (b + 1)) return;
  const int i = (int)(t / (b + 1)), q = (int)(t % (b + 1));
  const size_t ld = (size_t)band_ld(b);
  Ub[(size_t)i * ld + q] = (i + q < N) ? Lb[(size_t)(i + q) * ld + (b - q)] : 0.0;
}

enum SolveMode {
  FWD_U_FROM_V = 0,   // rhs_i = vin[u-dof(i)] / d,     out ty[i]
  FWD_P_FROM_T = 1,   // rhs_i = tp[i],                 out tp[i]
  FWD_P_FROM_V = 2,   // rhs_i = -vin[3i+2] / d,        out tp[i]
  BWD_U_TO_Z = 3,     // rhs_i = ty[i],                 out z[u-dof(i)]
  BWD_P_TO_Z = 4,     // rhs_i = tp[i],                 out z[3i+2]
  BWD_INPLACE = 5     // rhs_i = tp[i],                 out tp[i]
};

__device__ __forceinline__ int udof(int i) { return 3 * (i >> 1) + (i & 1); }

// Inverse of every kNB x kNB diagonal block of L (lower triangular), row-major,
// zero above the diagonal; rows past N are padded with the identity.
__global__ void k_diag_inverse(int N, int b, const double* __restrict__ Lb, double* __restrict__ Dinv) {
  __shared__ double Ld[kNB][kNB + 1];
  const int I = blockIdx.x, i0 = I * kNB, t = threadIdx.x;
  double* X = Dinv + (size_t)I * kNB * kNB;  // X[r * kNB + k]; column k written and read by thread k only
  const size_t W = (size_t)band_ld(b);
  for (int idx = t; idx < kNB * kNB; idx += blockDim.x) {
    const int r = idx / kNB, c = idx % kNB;
    double v = 0.0;
    if (c <= r) {
      if (i0 + r < N) {
        if (r - c <= b) v = Lb[(size_t)(i0 + r) * W + (b - (r - c))];
      } else {
        v = (r == c) ? 1.0 : 0.0;
      }
    }
    Ld[r][c] = v;
  }
  __syncthreads();
  if (t < kNB) {
    const int k = t;  // column k of the inverse: forward substitution on e_k
    for (int r = 0; r < kNB; ++r) {
      if (r < k) {
        X[r * kNB + k] = 0.0;
        continue;
      }
      double s = (r == k) ? 1.0 : 0.0;
      for (int j = k; j < r; ++j) s -= Ld[r][j] * X[j * kNB + k];
      X[r * kNB + k] = s / Ld[r][r];
    }
  }
}

// Blocked band triangular solve for kCols columns per CTA.
// Forward (L y = rhs): blocks ascending; row i of block I gets
//   s_i = sum_{j in [i-b, i0)} L[i][j] y_j,  y_I = Dinv_I (rhs_I - s_I).
// Backward (L^T x = rhs, rows of L^T in Ub): blocks descending;
//   s_i = sum_{j in (i0+kNB-1, i+b]} U[i][j] x_j,  x_I = Dinv_I^T (rhs_I - s_I).
template <int MODE, typename T>
__device__ __forceinline__ void band_solve_body(int N, int b, const T* __restrict__ band, const T* __restrict__ Dinv,
             const T* __restrict__ vin, const double* __restrict__ dsc, T* __restrict__ ty,
             T* __restrict__ tp, T* __restrict__ z, int ld, int c0, int ncols, int ring_mask) {
  constexpr bool kFwd = MODE <= FWD_P_FROM_V;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);              // [(ring_mask + 1) * kCols]
  T* tb = ring + (size_t)(ring_mask + 1) * kCols;        // [kNB * kCols]
  const int cbase = c0 + blockIdx.x * kCols;
  const int ncl = min(kCols, c0 + ncols - cbase);
  const int t = threadIdx.x;
  const int r = t / kKSplit, part = t % kKSplit;
  const int nblk = (N + kNB - 1) / kNB;
  const size_t W = (size_t)band_ld(b);

  auto read_rhs = [&](int i, int c) -> T {
    if (MODE == FWD_U_FROM_V) { const int rr = udof(i); return vin[(size_t)rr * ld + c] / (T)dsc[rr]; }
    if (MODE == FWD_P_FROM_T) return tp[(size_t)i * ld + c];
    if (MODE == FWD_P_FROM_V) { const int rr = 3 * i + 2; return -vin[(size_t)rr * ld + c] / (T)dsc[rr]; }
    if (MODE == BWD_U_TO_Z) return ty[(size_t)i * ld + c];
    return tp[(size_t)i * ld + c];
  };
  auto write_out = [&](int i, int c, T y) {
    if (MODE == FWD_U_FROM_V) ty[(size_t)i * ld + c] = y;
    else if (MODE == FWD_P_FROM_T || MODE == FWD_P_FROM_V) tp[(size_t)i * ld + c] = y;
    else if (MODE == BWD_U_TO_Z) z[(size_t)udof(i) * ld + c] = y;
    else z[(size_t)(3 * i + 2) * ld + c] = y;
  };
  auto block_of = [&](int bi) { return kFwd ? bi : (nblk - 1 - bi); };

  // right-hand side of this thread's row, prefetched one block ahead
  T rhs_next[kCols];
  {
    const int i = block_of(0) * kNB + r;
#pragma unroll
    for (int c = 0; c < kCols; ++c) rhs_next[c] = (part == 0 && i < N && c < ncl) ? read_rhs(i, cbase + c) : T(0);
  }
  for (int bi = 0; bi < nblk; ++bi) {
    const int I = block_of(bi);
    const int i0 = I * kNB;
    const int i = i0 + r;
    T rhs[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) rhs[c] = rhs_next[c];
    if (bi + 1 < nblk) {
      const int in = block_of(bi + 1) * kNB + r;
#pragma unroll
      for (int c = 0; c < kCols; ++c)
        rhs_next[c] = (part == 0 && in < N && c < ncl) ? read_rhs(in, cbase + c) : T(0);
    }
    // phase 1: band product with the rows outside this block
    T acc[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) acc[c] = T(0);
    if (i < N) {
      const T* Lrow = band + (size_t)i * W;
      int qs, qe;  // q in [qs, qe)
      if (kFwd) {
        qs = max(0, b - i);
        qe = b - r;
      } else {
        qs = kNB - r;
        qe = min(b, N - 1 - i) + 1;
      }
#pragma unroll 4
      for (int q = qs + part; q < qe; q += kKSplit) {
        const T l = Lrow[q];
        const int j = kFwd ? (i - b + q) : (i + q);
        const T* yr = ring + (size_t)(j & ring_mask) * kCols;
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] = fma(l, yr[c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kCols; ++c)
#pragma unroll
      for (int off = 1; off < kKSplit; off <<= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
    if (part == 0)
#pragma unroll
      for (int c = 0; c < kCols; ++c) tb[r * kCols + c] = (i < N) ? rhs[c] - acc[c] : T(0);
    __syncthreads();
    // phase 2: apply the inverse of the diagonal block (4 lanes per row)
    const T* D = Dinv + (size_t)I * kNB * kNB;
    T y[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) y[c] = T(0);
    if (kFwd) {
      for (int k = part; k <= r; k += kKSplit) {
        const T dv = D[r * kNB + k];
#pragma unroll
        for (int c = 0; c < kCols; ++c) y[c] = fma(dv, tb[k * kCols + c], y[c]);
      }
    } else {
      for (int k = r + part; k < kNB; k += kKSplit) {
        const T dv = D[k * kNB + r];
#pragma unroll
        for (int c = 0; c < kCols; ++c) y[c] = fma(dv, tb[k * kCols + c], y[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kCols; ++c)
#pragma unroll
      for (int off = 1; off < kKSplit; off <<= 1) y[c] += __shfl_xor_sync(0xffffffffu, y[c], off);
    if (part == 0 && i < N) {
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        ring[(size_t)(i & ring_mask) * kCols + c] = y[c];
        if (c < ncl) write_out(i, cbase + c, y[c]);
      }
    }
    __syncthreads();
  }
}

template <int MODE, typename T>
__global__ void __launch_bounds__(kSolveThreads)
k_band_solve(int N, int b, const T* __restrict__ band, const T* __restrict__ Dinv,
             const T* __restrict__ vin, const double* __restrict__ dsc, T* __restrict__ ty,
             T* __restrict__ tp, T* __restrict__ z, int ld, int c0, int ncols, int ring_mask) {
  band_solve_body<MODE, T>(N, b, band, Dinv, vin, dsc, ty, tp, z, ld, c0, ncols, ring_mask);
}

__host__ __device__ inline int ring_rows(int b) {
  int r = 1;
  while (r < b + kNB + 1) r <<= 1;
  return r;
}


// ---- TMA-staged variant --------------------------------------------------------
// The band rows of the next block are copied into shared memory by the bulk-copy
// engine (cp.async.bulk, completion on an mbarrier) while the current block is
// processed: two buffers, so the FP pipes never wait on band loads from L2. The
// band arrays are padded to a multiple of 64 rows, so every copy is one whole,
// 16-byte aligned block of NB rows. The diagonal-block inverses of NB-row blocks
// are the NB x NB diagonal sub-blocks of the 64-row inverses (the inverse of a
// block lower-triangular matrix has the inverted diagonal blocks on its diagonal).

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// One arrival that announces `bytes` of bulk-copy traffic for the current phase.
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of *bar for at most ~budget SM cycles; false on timeout. The clock
// is checked before every probe, so a budget of a cycle or two runs out before the first
// probe even when the copy has already landed (the failure-detection test relies on it).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  for (;;) {
    if (clock64() - t0 >= budget) return false;
    if (mbar_try_wait(bar, parity)) return true;
  }
}

constexpr long long kWaitBudget = 4000000000LL;  // ~2 s at 2 GHz

// Budget of the first wait of every block (the one that can report a timeout). Equal to
// kWaitBudget unless a test shortens it with biot_debug_set_wait_budget; the waits that drain
// copies still in flight before a CTA exits always keep the full kWaitBudget, so no CTA
// releases shared memory that a bulk copy is still writing.
__constant__ long long c_first_wait_budget = kWaitBudget;

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Ring rows R of the TMA-staged body, which indexes its ring modulo R (any R): phase 1 of a
// block reads the b rows before (forward) or after (backward) it, plus at most VQ - 1 below an
// aligned start, so R >= b + NB + 8 keeps every row it needs and, with each row stored at slots
// j mod R and j mod R + R, keeps every read window contiguous inside the 2 R slots.
__host__ __device__ constexpr int tma_ring_rows(int b, int nb) { return b + nb + 8; }

template <typename T, int NB>
__host__ __device__ inline size_t tma_smem_bytes(int b) {
  return 64 + 2 * align16((size_t)NB * band_ld(b) * sizeof(T)) + 2 * align16((size_t)NB * NB * sizeof(T)) +
         2 * (size_t)tma_ring_rows(b, NB) * kCols * sizeof(T) + (size_t)NB * kCols * sizeof(T);
}

// Compact inverses of the NB-row diagonal blocks, [block][NB][NB], taken from the
// 64-row inverses (diagonal sub-blocks).
template <typename T>
__global__ void k_extract_dnb(const T* __restrict__ D64, int N, int nb, T* __restrict__ out) {
  const int nblk = (N + nb - 1) / nb;
  const long long tot = (long long)nblk * nb * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t / (nb * nb)), rk = (int)(t % (nb * nb)), r = rk / nb, k = rk % nb;
    const int i0 = I * nb, o = i0 % 64;
    out[t] = D64[(size_t)(i0 / 64) * 64 * 64 + (size_t)(o + r) * 64 + o + k];
  }
}

template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using V = float4;
  static constexpr int n = 4;
  __device__ __forceinline__ static void get(const V& v, float* out) { out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w; }
};
template <> struct Vec16<double> {
  using V = double2;
  static constexpr int n = 2;
  __device__ __forceinline__ static void get(const V& v, double* out) { out[0] = v.x; out[1] = v.y; }
};

// Sum of a and b over the KS lanes of a row group (KS a power of two, 2 <= KS <= 32),
// transposed: lane `part` receives the sum of a when part is even and of b when odd,
// with one add per lane per round instead of two.
template <int KS, typename T>
__device__ __forceinline__ T reduce_pair(T a, T b, int part) {
  const bool odd = part & 1;
  T keep = odd ? b : a;
  keep += __shfl_xor_sync(0xffffffffu, odd ? a : b, 1);
#pragma unroll
  for (int off = 2; off < KS; off <<= 1) keep += __shfl_xor_sync(0xffffffffu, keep, off);
  return keep;
}

template <int MODE, typename T, int NB, int THREADS>
__device__ __forceinline__ void
band_solve_tma_body(int N, int b, const T* __restrict__ band, const T* __restrict__ Dnb, const T* __restrict__ vin,
                    const double* __restrict__ dsq, T* __restrict__ ty, T* __restrict__ tp, T* __restrict__ z, int ld,
                    int c0, int ncols, int ring_mask, int strip_rows, int blk, int32_t* __restrict__ err) {
  constexpr bool kFwd = MODE <= FWD_P_FROM_V;
  constexpr int KS = THREADS / NB;  // lanes sharing one row
  constexpr int VQ = Vec16<T>::n;   // band entries per 16-byte load
  static_assert(THREADS % NB == 0 && KS <= 32 && (KS & (KS - 1)) == 0 && KS >= 2, "bad split");
  static_assert(THREADS >= 128 && NB % 4 == 0 && 64 % NB == 0, "phase 2 maps NB/4 rows to each of 4 warps");
  static_assert(kCols == 2, "the ring rows are read as pairs");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lb = band_ld(b);
  const int R = ring_mask + 1;   // the ring holds every row twice: slots j mod R and j mod R + R
  if (strip_rows > 0) {
    // strip blockIdx.y of a block-diagonal band matrix (N = strip_rows rows each, a multiple
    // of NB): its own band rows, block inverses and rows of the in-place buffer
    const size_t r0 = (size_t)blockIdx.y * strip_rows;
    band += r0 * lb;
    Dnb += r0 * NB;
    tp += r0 * ld;
  }
  const size_t bufb = align16((size_t)NB * lb * sizeof(T));
  constexpr size_t dbufb = align16((size_t)NB * NB * sizeof(T));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  auto buf = [&](int slot) { return reinterpret_cast<T*>(smem_raw + 64 + slot * bufb); };
  auto dbuf = [&](int slot) { return reinterpret_cast<T*>(smem_raw + 64 + 2 * bufb + slot * dbufb); };
  T* ring = reinterpret_cast<T*>(smem_raw + 64 + 2 * bufb + 2 * dbufb);  // [2R][kCols]
  T* tb = ring + (size_t)2 * R * kCols;
  const int cbase = c0 + blockIdx.x * kCols;
  const int ncl = min(kCols, c0 + ncols - cbase);
  const int t = threadIdx.x;
  const int r = t / KS, part = t % KS;
  const int nblk = (N + NB - 1) / NB;
  const uint32_t bytes = (uint32_t)((size_t)NB * lb * sizeof(T));
  constexpr uint32_t dbytes = (uint32_t)(NB * NB * sizeof(T));

  auto read_rhs = [&](int i, int c) -> T {
    if (MODE == FWD_U_FROM_V) { const int rr = udof(i); return vin[(size_t)rr * ld + c] * (T)dsq[rr]; }
    if (MODE == FWD_P_FROM_T) return tp[(size_t)i * ld + c];
    if (MODE == FWD_P_FROM_V) { const int rr = 3 * i + 2; return -vin[(size_t)rr * ld + c] * (T)dsq[rr]; }
    if (MODE == BWD_U_TO_Z) return ty[(size_t)i * ld + c];
    return tp[(size_t)i * ld + c];
  };
  auto write_out = [&](int i, int c, T y) {
    if (MODE == FWD_U_FROM_V) ty[(size_t)i * ld + c] = y;
    else if (MODE == FWD_P_FROM_T || MODE == FWD_P_FROM_V) tp[(size_t)i * ld + c] = y;
    else if (MODE == BWD_U_TO_Z) z[(size_t)udof(i) * ld + c] = y;
    else if (MODE == BWD_INPLACE) tp[(size_t)i * ld + c] = y;
    else z[(size_t)(3 * i + 2) * ld + c] = y;
  };
  auto block_of = [&](int bi) { return kFwd ? bi : (nblk - 1 - bi); };
  auto issue = [&](int bi) {
    const int I = block_of(bi);
    mbar_expect(&bar[bi & 1], bytes + dbytes);
    bulk_copy(buf(bi & 1), band + (size_t)I * NB * lb, bytes, &bar[bi & 1]);
    bulk_copy(dbuf(bi & 1), Dnb + (size_t)I * NB * NB, dbytes, &bar[bi & 1]);
  };

  // rows outside 0..N-1 read by the vectorised loop meet zero band entries: keep them finite
  for (int k = t; k < 2 * R * kCols; k += THREADS) ring[k] = T(0);
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0) {
    issue(0);
    if (nblk > 1) issue(1);
  }
  // lane `part` of a row holds the right-hand side of column `part` (part < kCols)
  T rhs_next;
  {
    const int i = block_of(0) * NB + r;
    rhs_next = (part < ncl && i < N) ? read_rhs(i, cbase + part) : T(0);
  }
  for (int bi = 0; bi < nblk; ++bi) {
    const int I = block_of(bi);
    const int i0 = I * NB;
    const int i = i0 + r;
    const T rhs = rhs_next;
    if (bi + 1 < nblk) {
      const int in = block_of(bi + 1) * NB + r;
      rhs_next = (part < ncl && in < N) ? read_rhs(in, cbase + part) : T(0);
    }
    // band rows of this block: wait for the bulk copy (bounded)
    const bool ok = mbar_wait_bounded(&bar[bi & 1], (uint32_t)((bi >> 1) & 1), c_first_wait_budget);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicExch(err, 1);
        // let copies still in flight land before the CTA's shared memory is released
        mbar_wait_bounded(&bar[bi & 1], (uint32_t)((bi >> 1) & 1), kWaitBudget);
        if (bi + 1 < nblk) mbar_wait_bounded(&bar[(bi + 1) & 1], (uint32_t)(((bi + 1) >> 1) & 1), kWaitBudget);
      }
      __syncthreads();
      return;
    }
    const T* rows = buf(bi & 1);
    T acc0 = T(0), acc1 = T(0);
    if (i < N) {
      // off-block band entries q in [qs, qe): forward j = i - b + q < i0, backward j = i + q > i0 + NB - 1.
      // blk > 0: the factor of a block-tridiagonal matrix with blk x blk blocks, whose row i has no
      // entries left of block i / blk - 1 (forward) and whose column i none below block i / blk + 1
      // (backward): those band entries are exact zeros and are skipped.
      int qs = kFwd ? max(0, b - i) : NB - r;
      int qe = kFwd ? b - r : min(b, N - 1 - i) + 1;
      if (blk > 0) {
        if (kFwd) qs = max(qs, max(0, (i / blk - 1) * blk) - (i - b));
        else qe = min(qe, (i / blk + 2) * blk - i);
      }
      if (qs < qe && sizeof(T) == 4) {
        // FP32: one band entry per lane and step, so consecutive lanes read consecutive band
        // words and ring rows (both columns of a row as one 8-byte load): no bank conflicts.
        // Chunks of VQ entries per lane (below) read the ring at a 4-row stride across lanes,
        // an 8-way conflict that FP32's short multiply-adds cannot hide (FP64's can).
        const T* Lrow = rows + (size_t)r * lb;
        int s0 = (kFwd ? (i - b + qs) : (i + qs)) % R;
        if (s0 < 0) s0 += R;
        s0 -= qs;  // ring slot of entry q: s0 + q, below 2 R for q < qe
        // Four entries' loads go out before their multiply-adds, into four accumulator pairs:
        // with one warp per SM sub-partition nothing else hides the shared-memory latency.
        using V2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
        const V2* ring2 = reinterpret_cast<const V2*>(ring);
        T a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = T(0);
        int q = qs + part;
        for (; q + 3 * KS < qe; q += 4 * KS) {
          T l[4];
          V2 y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            l[u] = Lrow[q + u * KS];
            y[u] = ring2[s0 + q + u * KS];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            a[2 * u] = fma(l[u], y[u].x, a[2 * u]);
            a[2 * u + 1] = fma(l[u], y[u].y, a[2 * u + 1]);
          }
        }
        for (; q < qe; q += KS) {
          const T l0 = Lrow[q];
          const V2 y0 = ring2[s0 + q];
          a[0] = fma(l0, y0.x, a[0]);
          a[1] = fma(l0, y0.y, a[1]);
        }
        acc0 = (a[0] + a[2]) + (a[4] + a[6]);
        acc1 = (a[1] + a[3]) + (a[5] + a[7]);
      } else if (qs < qe) {
        const T* Lrow = rows + (size_t)r * lb;
        const int qa = qs & ~(VQ - 1);  // 16-byte aligned start
        int s0 = (kFwd ? (i - b + qa) : (i + qa)) % R;
        if (s0 < 0) s0 += R;
        // Forward: entries below qs are zero (rows j < 0), entries from qe on are inside the
        // block and are masked. Backward: entries below qs are inside the block and masked,
        // entries past qe are zero (rows j >= N, row padding).
#pragma unroll 2
        for (int q4 = qa + part * VQ; q4 < qe; q4 += KS * VQ) {
          T l[VQ];
          Vec16<T>::get(*reinterpret_cast<const typename Vec16<T>::V*>(Lrow + q4), l);
          if (kFwd ? (q4 + VQ > qe) : (q4 < qs)) {
#pragma unroll
            for (int k = 0; k < VQ; ++k)
              if (kFwd ? (q4 + k >= qe) : (q4 + k < qs)) l[k] = T(0);
          }
          const T* y = ring + (size_t)(s0 + (q4 - qa)) * kCols;
#pragma unroll
          for (int k = 0; k < VQ; ++k) {
            acc0 = fma(l[k], y[2 * k], acc0);
            acc1 = fma(l[k], y[2 * k + 1], acc1);
          }
        }
      }
    }
    // transposed reduction over the row's KS lanes: lane `part` ends with column part & 1
    const T s1 = reduce_pair<KS>(acc0, acc1, part);
    if (part < kCols) tb[r * kCols + part] = (i < N) ? rhs - s1 : T(0);
    __syncthreads();
    // diagonal block (its NB x NB inverse arrived with the band rows, zero outside the
    // triangle) on warps 0..3, one per SM sub-partition: warp w owns rows w*NB/4 ..
    // w*NB/4 + NB/4 - 1; lane = o * P2L + h, output o = (row, column), h splits the terms
    if (t < 128) {
      constexpr int P2L = 64 / NB;
      const int w = t >> 5, lane = t & 31;
      const int o = lane / P2L, h = lane % P2L;
      const int r2 = w * (NB / 4) + (o >> 1), c2 = o & 1;
      const T* D = dbuf(bi & 1);
      T y = T(0);
      if constexpr (sizeof(T) == 4) {
        // the inverse is lower triangular: forward rows stop at k = r2, backward columns start
        // there (skipping exact zeros leaves every sum bitwise unchanged). Measured faster in
        // FP32; in FP64 the fully unrolled loop below keeps the latency-bound chains shorter.
        if (kFwd) {
          for (int k = h; k <= r2; k += P2L) y = fma(D[r2 * NB + k], tb[k * kCols + c2], y);
        } else {
          for (int k = r2 + ((h - r2) & (P2L - 1)); k < NB; k += P2L) y = fma(D[k * NB + r2], tb[k * kCols + c2], y);
        }
      } else {
#pragma unroll
        for (int k = h; k < NB; k += P2L) y = fma(kFwd ? D[r2 * NB + k] : D[k * NB + r2], tb[k * kCols + c2], y);
      }
#pragma unroll
      for (int off = 1; off < P2L; off <<= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
      const int i2 = i0 + r2;
      if (h == 0 && i2 < N) {
        const int sl = i2 % R;
        ring[(size_t)sl * kCols + c2] = y;
        ring[(size_t)(sl + R) * kCols + c2] = y;
        if (c2 < ncl) write_out(i2, cbase + c2, y);
      }
    }
    __syncthreads();
    // both buffers of slot bi & 1 are free again: prefetch block bi + 2 into them
    if (t == 0 && bi + 2 < nblk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(bi + 2);
    }
  }
}

template <int MODE, typename T, int NB, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_band_solve_tma(int N, int b, const T* __restrict__ band, const T* __restrict__ Dnb, const T* __restrict__ vin,
                 const double* __restrict__ dsq, T* __restrict__ ty, T* __restrict__ tp, T* __restrict__ z, int ld,
                 int c0, int ncols, int ring_mask, int strip_rows, int blk, int32_t* __restrict__ err) {
  band_solve_tma_body<MODE, T, NB, THREADS>(N, b, band, Dnb, vin, dsq, ty, tp, z, ld, c0, ncols, ring_mask, strip_rows,
                                            blk, err);
}

// ---- row-per-lane in-place band solve for narrow bands (strip interiors) ----
//
// Lane (r, cp) of a warp owns row r of a 16-row block and column pair cp (two of the warp's
// four columns) and runs that row's whole off-block band product itself: no lane reductions,
// and the block's 16 x 16 inverse costs 16 multiply-adds per column. The CTA's warps take
// consecutive column groups and share each block's band rows (one bulk copy per row into rows
// whose byte stride is 16 mod 32, so the 16 rows fall two by two on the bank pairs) and its
// inverse (stored with row stride 17 for conflict-free row and column access); each warp keeps
// its own solution ring. For small half-bands this issues far fewer FP64 instructions per
// band entry than the split-row kernel.
constexpr int kRowsNB = 16;
constexpr int kRowsCols = 4;        // columns per warp
constexpr int kRowsDs = kRowsNB + 1;  // row stride of the stored block inverses

template <typename T> __host__ __device__ inline int rows_stride(int b) {
  int s = band_ld(b);
  if ((s * (int)sizeof(T)) % 32 == 0) s += 16 / (int)sizeof(T);
  return s;
}
__host__ __device__ inline int rows_ring(int b) {
  int r = 2;
  while (r < b + kRowsNB + 1) r <<= 1;
  return r;
}
template <typename T> size_t rows_smem_bytes(int b, int warps) {
  const size_t bandb = align16((size_t)kRowsNB * rows_stride<T>(b) * sizeof(T));
  const size_t dbb = align16((size_t)kRowsNB * kRowsDs * sizeof(T));
  const size_t ring = (size_t)warps * 2 * rows_ring(b) * kRowsCols * sizeof(T);
  const size_t tb = (size_t)warps * kRowsNB * kRowsCols * sizeof(T);
  return 64 + 2 * bandb + 2 * dbb + ring + tb;
}

// 16 x 16 diagonal-block inverses with row stride 17, from the 64 x 64 ones.
template <typename T>
__global__ void k_extract_dnb17(const T* __restrict__ D64, int N, T* __restrict__ out) {
  const int nblk = (N + kRowsNB - 1) / kRowsNB;
  const long long tot = (long long)nblk * kRowsNB * kRowsDs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t / (kRowsNB * kRowsDs)), rk = (int)(t % (kRowsNB * kRowsDs));
    const int r = rk / kRowsDs, k = rk % kRowsDs;
    const int i0 = I * kRowsNB, o = i0 % 64;
    out[t] = k < kRowsNB ? D64[(size_t)(i0 / 64) * 64 * 64 + (size_t)(o + r) * 64 + o + k] : T(0);
  }
}

template <int MODE, typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_band_solve_rows(int N, int b, const T* __restrict__ band, const T* __restrict__ Dnb, T* __restrict__ buf, int ld,
                  int c0, int ncols, int ring_mask, int strip_rows, int32_t* __restrict__ err) {
  constexpr bool kFwd = MODE <= FWD_P_FROM_V;
  constexpr int NB = kRowsNB;
  static_assert(MODE == FWD_P_FROM_T || MODE == BWD_INPLACE, "in-place solves only");
  using V2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lb = band_ld(b);
  const int S = rows_stride<T>(b);
  const int R = ring_mask + 1;
  if (strip_rows > 0) {
    const size_t r0 = (size_t)blockIdx.y * strip_rows;
    band += r0 * lb;
    Dnb += (r0 / NB) * NB * kRowsDs;
    buf += r0 * ld;
  }
  const size_t bandb = align16((size_t)NB * S * sizeof(T));
  constexpr size_t dbb = align16((size_t)NB * kRowsDs * sizeof(T));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  auto rows_at = [&](int slot) { return reinterpret_cast<T*>(smem_raw + 64 + slot * bandb); };
  auto d_at = [&](int slot) { return reinterpret_cast<T*>(smem_raw + 64 + 2 * bandb + slot * dbb); };
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  T* rings = reinterpret_cast<T*>(smem_raw + 64 + 2 * bandb + 2 * dbb);
  T* ring = rings + (size_t)warp * 2 * R * kRowsCols;                                 // [2R][4]
  T* tb = rings + (size_t)WARPS * 2 * R * kRowsCols + (size_t)warp * NB * kRowsCols;  // [NB][4]
  const int r = lane % NB, cp = lane / NB;
  const int ca = c0 + (blockIdx.x * WARPS + warp) * kRowsCols + 2 * cp;  // the lane's columns ca, ca + 1
  const bool v0 = ca < c0 + ncols, v1 = ca + 1 < c0 + ncols;
  const int nblk = (N + NB - 1) / NB;
  const uint32_t rowbytes = (uint32_t)(lb * sizeof(T));
  constexpr uint32_t dbytes = (uint32_t)(NB * kRowsDs * sizeof(T));
  auto block_of = [&](int bi) { return kFwd ? bi : (nblk - 1 - bi); };
  auto issue = [&](int bi) {
    const int I = block_of(bi), sl = bi & 1;
    mbar_expect(&bar[sl], NB * rowbytes + dbytes);
    for (int k = 0; k < NB; ++k) bulk_copy(rows_at(sl) + (size_t)k * S, band + ((size_t)I * NB + k) * lb, rowbytes, &bar[sl]);
    bulk_copy(d_at(sl), Dnb + (size_t)I * NB * kRowsDs, dbytes, &bar[sl]);
  };
  auto read_rhs = [&](int i, T& a0, T& a1) {
    a0 = (v0 && i < N) ? buf[(size_t)i * ld + ca] : T(0);
    a1 = (v1 && i < N) ? buf[(size_t)i * ld + ca + 1] : T(0);
  };

  // rows outside 0..N-1 meet zero band entries: keep the ring finite
  for (int k = lane; k < 2 * R * kRowsCols; k += 32) ring[k] = T(0);
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0) {
    issue(0);
    if (nblk > 1) issue(1);
  }
  T rn0, rn1;
  read_rhs(block_of(0) * NB + r, rn0, rn1);
  for (int bi = 0; bi < nblk; ++bi) {
    const int I = block_of(bi);
    const int i = I * NB + r;
    const T rh0 = rn0, rh1 = rn1;
    if (bi + 1 < nblk) read_rhs(block_of(bi + 1) * NB + r, rn0, rn1);
    const bool ok = mbar_wait_bounded(&bar[bi & 1], (uint32_t)((bi >> 1) & 1), c_first_wait_budget);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicExch(err, 1);
        // let copies still in flight land before the CTA's shared memory is released
        mbar_wait_bounded(&bar[bi & 1], (uint32_t)((bi >> 1) & 1), kWaitBudget);
        if (bi + 1 < nblk) mbar_wait_bounded(&bar[(bi + 1) & 1], (uint32_t)(((bi + 1) >> 1) & 1), kWaitBudget);
      }
      __syncthreads();
      return;
    }
    // off-block band product of row i: forward j = i - b + q < i0, backward j = i + q > i0 + NB - 1
    T acc0 = T(0), acc1 = T(0);
    if (i < N) {
      const T* Lrow = rows_at(bi & 1) + (size_t)r * S;
      const int qs = kFwd ? max(0, b - i) : NB - r;
      const int qe = kFwd ? b - r : min(b, N - 1 - i) + 1;
      const T* y = ring + (size_t)((kFwd ? (i - b) : i) & ring_mask) * kRowsCols + 2 * cp;
#pragma unroll 4
      for (int q = qs; q < qe; ++q) {
        const T l = Lrow[q];
        const V2 yy = *reinterpret_cast<const V2*>(y + (size_t)q * kRowsCols);
        acc0 = fma(l, yy.x, acc0);
        acc1 = fma(l, yy.y, acc1);
      }
    }
    tb[r * kRowsCols + 2 * cp] = (i < N) ? rh0 - acc0 : T(0);
    tb[r * kRowsCols + 2 * cp + 1] = (i < N) ? rh1 - acc1 : T(0);
    __syncwarp();
    // diagonal block: y = D_I t (D_I's inverse rows at stride 17, zero outside the triangle)
    const T* D = d_at(bi & 1);
    T y0 = T(0), y1 = T(0);
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const T dv = kFwd ? D[r * kRowsDs + k] : D[k * kRowsDs + r];
      const V2 tt = *reinterpret_cast<const V2*>(tb + k * kRowsCols + 2 * cp);
      y0 = fma(dv, tt.x, y0);
      y1 = fma(dv, tt.y, y1);
    }
    if (i < N) {
      const int sl = i & ring_mask;
      *reinterpret_cast<V2*>(ring + (size_t)sl * kRowsCols + 2 * cp) = V2{y0, y1};
      *reinterpret_cast<V2*>(ring + (size_t)(sl + R) * kRowsCols + 2 * cp) = V2{y0, y1};
      if (v0) buf[(size_t)i * ld + ca] = y0;
      if (v1) buf[(size_t)i * ld + ca + 1] = y1;
    }
    __syncthreads();  // every warp is done with stage bi & 1 and with this block's tb
    if (t == 0 && bi + 2 < nblk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(bi + 2);
    }
  }
}

template <int MODE, typename T, int WARPS>
static void launch_rows(biot_ctx* ctx, int N, int b, const T* band, const T* Dnb17, T* buf, int ld, int c0, int ncols,
                        int nstrips) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_band_solve_rows<MODE, T, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  const dim3 grid(div_up(ncols, WARPS * kRowsCols), nstrips);
  BIOT_LAUNCH((k_band_solve_rows<MODE, T, WARPS>), grid, WARPS * 32, rows_smem_bytes<T>(b, WARPS), ctx->stream, N, b,
              band, Dnb17, buf, ld, c0, ncols, rows_ring(b) - 1, N, ctx->status);
}

// Batched form (instance = blockIdx.z, FP32): the same solve on each active instance's
// factors, compact block inverses and Krylov vector j (V_j in, Z_j out).
constexpr int kBatchNB = 32;
constexpr int kBatchThreads = 256;
template <int MODE>
__global__ void __launch_bounds__(kBatchThreads) kb_band_solve_tma(const InstDev* __restrict__ tab, int j) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0 || (int)blockIdx.x * kCols >= I.nf) return;
  const size_t vs = (size_t)I.n_dof * I.wcap;
  const bool u = (MODE == FWD_U_FROM_V || MODE == BWD_U_TO_Z);
  const int N = u ? 2 * I.n_nodes : I.n_nodes;
  const int b = u ? I.band_u : I.band_p;
  const float* band = (MODE == FWD_U_FROM_V) ? I.Lu : (MODE == BWD_U_TO_Z) ? I.Uu : (MODE == BWD_P_TO_Z) ? I.Up : I.Lp;
  const float* Dnb = u ? I.dnbu : I.dnbp;
  band_solve_tma_body<MODE, float, kBatchNB, kBatchThreads>(N, b, band, Dnb, I.V + j * vs, I.dsq, I.tu, I.tp,
                                                            I.Z + j * vs, I.wcap, I.c0, I.nf, tma_ring_rows(b, kBatchNB) - 1, 0,
                                                            0, I.status);
}

__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = (float)src[k];
}

// Full band Cholesky of an SPD band matrix held in Lb (in place).
biot_status band_cholesky(biot_ctx* ctx, int N, int b, double* Lb) {
  BIOT_CU(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), ctx->stream));
  const long long tri = (long long)b * (b + 1) / 2;
  const int ublocks = (int)std::min<long long>((tri + 255) / 256, 2048);
  for (int j0 = 0; j0 < N; j0 += kPanel) {
    const int np = std::min(kPanel, N - j0);
    BIOT_LAUNCH(k_chol_panel, 1, 256, 0, ctx->stream, N, b, j0, np, Lb, ctx->status);
    if (j0 + np < N) BIOT_LAUNCH(k_chol_trailing, ublocks, 256, 0, ctx->stream, N, b, j0, np, Lb, ctx->status);
  }
  BIOT_CU(ctx, cudaGetLastError());
  int32_t st = 0;
  BIOT_CU(ctx, cudaMemcpyAsync(&st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  if (st != 0) return fail(ctx, BIOT_E_CUDA, "band Cholesky: non-positive pivot at row %d", st - 1);
  return BIOT_OK;
}

}  // namespace

// Natural-order band factors of A and S (FP64, and FP32 copies for the reduced-precision
// sweeps) with their default solve variants and block inverses.
static biot_status plain_band_setup(biot_ctx* ctx) {
  const int nn = ctx->n_nodes;
  const int bu = ctx->band_u, bp = ctx->band_p;
  if (bu + kNB > 8192) return fail(ctx, BIOT_E_INVALID, "mesh too large for the band solver (half-band %d)", bu);
  // band rows padded to a multiple of 64 (whole-block bulk copies), zero beyond N
  const size_t su = (size_t)div_up(2 * nn, 64) * 64 * band_ld(bu), sp = (size_t)div_up(nn, 64) * 64 * band_ld(bp);
  if (!ctx->Lu) {
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Lu, sizeof(double) * su));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Uu, sizeof(double) * su));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Lp, sizeof(double) * sp));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Up, sizeof(double) * sp));
    const size_t nbu = (size_t)div_up(2 * nn, kNB), nbp = (size_t)div_up(nn, kNB);
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Du, sizeof(double) * nbu * kNB * kNB));
    BIOT_TRY(dalloc(ctx, (void**)&ctx->Dp, sizeof(double) * nbp * kNB * kNB));
  }
  cudaStream_t s = ctx->stream;
  BIOT_CU(ctx, cudaMemsetAsync(ctx->Lu, 0, sizeof(double) * su, s));
  BIOT_CU(ctx, cudaMemsetAsync(ctx->Lp, 0, sizeof(double) * sp, s));
  BIOT_CU(ctx, cudaMemsetAsync(ctx->Uu, 0, sizeof(double) * su, s));
  BIOT_CU(ctx, cudaMemsetAsync(ctx->Up, 0, sizeof(double) * sp, s));
  BIOT_LAUNCH(k_band_extract_u, div_up(2 * nn, 256), 256, 0, s, nn, bu, ctx->rowptr, ctx->col, ctx->val, ctx->Lu);
  BIOT_LAUNCH(k_band_extract_p, div_up(nn, 256), 256, 0, s, nn, bp, ctx->rowptr, ctx->col, ctx->val, ctx->Lp);
  BIOT_TRY(band_cholesky(ctx, 2 * nn, bu, ctx->Lu));
  BIOT_TRY(band_cholesky(ctx, nn, bp, ctx->Lp));
  BIOT_LAUNCH(k_band_transpose, div_up((long long)2 * nn * (bu + 1), 256), 256, 0, s, 2 * nn, bu, ctx->Lu, ctx->Uu);
  BIOT_LAUNCH(k_band_transpose, div_up((long long)nn * (bp + 1), 256), 256, 0, s, nn, bp, ctx->Lp, ctx->Up);
  BIOT_LAUNCH(k_diag_inverse, div_up(2 * nn, kNB), 256, 0, s, 2 * nn, bu, ctx->Lu, ctx->Du);
  BIOT_LAUNCH(k_diag_inverse, div_up(nn, kNB), 256, 0, s, nn, bp, ctx->Lp, ctx->Dp);
  if (ctx->prm.precision != BIOT_FP64) {
    // reduced-precision sweep: the exact FP64 factors rounded to FP32
    const size_t du = (size_t)div_up(2 * nn, kNB) * kNB * kNB, dp = (size_t)div_up(nn, kNB) * kNB * kNB;
    if (!ctx->lp.Lu) {
      BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.Lu, sizeof(float) * su));
      BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.Uu, sizeof(float) * su));
      BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.Du, sizeof(float) * du));
      BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.Lp, sizeof(float) * sp));
      BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.Up, sizeof(float) * sp));
      BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.Dp, sizeof(float) * dp));
    }
    const int g = 1024;
    BIOT_LAUNCH(k_to_f32, g, 256, 0, s, ctx->Lu, ctx->lp.Lu, su);
    BIOT_LAUNCH(k_to_f32, g, 256, 0, s, ctx->Uu, ctx->lp.Uu, su);
    BIOT_LAUNCH(k_to_f32, g, 256, 0, s, ctx->Du, ctx->lp.Du, du);
    BIOT_LAUNCH(k_to_f32, g, 256, 0, s, ctx->Lp, ctx->lp.Lp, sp);
    BIOT_LAUNCH(k_to_f32, g, 256, 0, s, ctx->Up, ctx->lp.Up, sp);
    BIOT_LAUNCH(k_to_f32, g, 256, 0, s, ctx->Dp, ctx->lp.Dp, dp);
  }
  BIOT_CU(ctx, cudaGetLastError());
  ctx->lp.tile_ok[0] = ctx->lp.tile_ok[1] = 0;  // factors changed: rebuild the tiles on demand
  ctx->lp.bdnb_ok = 0;
  for (int pi = 0; pi < 2; ++pi) {
    ctx->band_var_u[pi] = band_variant_default(pi == 0, bu);
    ctx->band_var_p[pi] = band_variant_default(pi == 0, bp);
    ctx->dnb_nb_u[pi] = ctx->dnb_nb_p[pi] = 0;  // factors changed: rebuild the compact inverses
    if (pi == 1 && ctx->prm.precision == BIOT_FP64) continue;
    BIOT_TRY(ensure_dnb(ctx, pi == 0, true, ctx->band_var_u[pi]));
    BIOT_TRY(ensure_dnb(ctx, pi == 0, false, ctx->band_var_p[pi]));
  }
  return BIOT_OK;
}

// Meshes above this size skip the natural-order factors when their blocks are substructured:
// at n = 1024 A's band factor alone would hold 35 GB in FP64 and cost about 9 TFLOP to form.
constexpr int kPlainBandMaxN = 512;

biot_status band_setup(biot_ctx* ctx, int kind) {
  ctx->plain_band = sub_strips(ctx) < 2 || ctx->n <= kPlainBandMaxN;
  if (ctx->plain_band) {
    BIOT_TRY(plain_band_setup(ctx));
  } else {
    for (int pi = 0; pi < 2; ++pi) ctx->band_var_u[pi] = ctx->band_var_p[pi] = -1;
  }
  BIOT_TRY(sub_setup(ctx));
  ctx->precond = kind;
  return BIOT_OK;
}

template <typename T> struct BandBufs;
template <> struct BandBufs<double> {
  static double* tu(biot_ctx* c) { return c->tu; }
  static double* tp(biot_ctx* c) { return c->tp; }
  static const double* Lu(biot_ctx* c) { return c->Lu; }
  static const double* Uu(biot_ctx* c) { return c->Uu; }
  static const double* Du(biot_ctx* c) { return c->Du; }
  static const double* Lp(biot_ctx* c) { return c->Lp; }
  static const double* Up(biot_ctx* c) { return c->Up; }
  static const double* Dp(biot_ctx* c) { return c->Dp; }
  static const double* Dnbu(biot_ctx* c) { return (const double*)c->dnb_u[0]; }
  static const double* Dnbp(biot_ctx* c) { return (const double*)c->dnb_p[0]; }
};
template <> struct BandBufs<float> {
  static float* tu(biot_ctx* c) { return c->lp.tu; }
  static float* tp(biot_ctx* c) { return c->lp.tp; }
  static const float* Lu(biot_ctx* c) { return c->lp.Lu; }
  static const float* Uu(biot_ctx* c) { return c->lp.Uu; }
  static const float* Du(biot_ctx* c) { return c->lp.Du; }
  static const float* Lp(biot_ctx* c) { return c->lp.Lp; }
  static const float* Up(biot_ctx* c) { return c->lp.Up; }
  static const float* Dp(biot_ctx* c) { return c->lp.Dp; }
  static const float* Dnbu(biot_ctx* c) { return (const float*)c->dnb_u[1]; }
  static const float* Dnbp(biot_ctx* c) { return (const float*)c->dnb_p[1]; }
};

template <int MODE, typename T, int NB, int THREADS>
static void launch_tma_raw(biot_ctx* ctx, int N, int b, const T* band, const T* Dnb, const T* vin, T* ty, T* tp, T* z,
                           int ld, int c0, int ncols, int nstrips, int strip_rows, int blk = 0) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_band_solve_tma<MODE, T, NB, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_set = true;
  }
  const int rr = tma_ring_rows(b, NB);
  const size_t smem = tma_smem_bytes<T, NB>(b);
  const dim3 grid(div_up(ncols, kCols), nstrips);
  BIOT_LAUNCH((k_band_solve_tma<MODE, T, NB, THREADS>), grid, THREADS, smem, ctx->stream, N, b, band, Dnb, vin,
              ctx->dsq, ty, tp, z, ld, c0, ncols, rr - 1, strip_rows, blk, ctx->status);
}

template <int MODE, typename T, int NB, int THREADS>
static void launch_tma(biot_ctx* ctx, int N, int b, const T* band, const T* Dinv, const T* vin, T* z, int c0,
                       int ncols) {
  launch_tma_raw<MODE, T, NB, THREADS>(ctx, N, b, band, Dinv, vin, BandBufs<T>::tu(ctx), BandBufs<T>::tp(ctx), z,
                                       ctx->wcap, c0, ncols, 1, 0);
}

// ---- FP32 band solves on skewed block tiles ----
//
// For block I (rows i0 .. i0 + NB - 1) the band entries that couple it to rows already
// solved are stored as one dense NB x W tile, W = band_ld(b), aligned on the solution
// index j = o + jj:
//   forward  (L):   o = i0 - b rounded down to even, T[r][jj] = L[i0 + r][j] for
//                   i0 + r - b <= j < i0, j >= 0;
//   backward (L^T): o = i0 + NB, T[r][jj] = L^T[i0 + r][j] for j <= i0 + r + b, j < N;
// every other entry (outside the band, inside the diagonal block, past the matrix) is an
// explicit zero. The product of a tile with the solution window then needs no masks, and
// a lane's 16-byte chunk of the window (four solution rows, both columns) serves four tile
// rows at once, cutting the shared-memory reads per multiply-add to a quarter of the
// row-by-row kernel's.
constexpr int kTileNB = 32;
constexpr int kTileThreads = 256;
// Two stages: deeper pipelines measured no faster alone and slower beside the concurrent
// S solves of P2 (a smaller footprint lets two S-solve CTAs share an SM).
constexpr int kTileMaxStages = 2;

__host__ __device__ inline long long tile_origin(bool fwd, int i0, int b) {
  return fwd ? (long long)((i0 - b) & ~1) : (long long)i0 + kTileNB;
}

__global__ void k_band_to_tiles(const float* __restrict__ band, int N, int b, bool fwd, float* __restrict__ tiles) {
  const int W = band_ld(b);
  const long long per = (long long)kTileNB * W;
  const long long tot = (long long)((N + kTileNB - 1) / kTileNB) * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t / per), rem = (int)(t % per);
    const int r = rem / W, jj = rem % W;
    const int i0 = I * kTileNB, i = i0 + r;
    const long long j = tile_origin(fwd, i0, b) + jj;
    float v = 0.f;
    if (i < N && j >= 0 && j < N) {
      if (fwd) {
        if (j >= (long long)i - b && j < i0) v = band[(size_t)i * W + (size_t)(j - (i - b))];
      } else {
        if (j <= (long long)i + b && j >= i0 + kTileNB) v = band[(size_t)i * W + (size_t)(j - i)];
      }
    }
    tiles[t] = v;
  }
}

// Sum over a warp's 32 lanes of eight values per lane, transposed: lane l ends with the
// sum of value (l >> 2) & 7 after 4 + 2 + 1 + 1 + 1 adds.
__device__ __forceinline__ float reduce8(const float (&v)[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  float u4[4], u2[2];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    u4[k] = (h16 ? v[k + 4] : v[k]) + __shfl_xor_sync(0xffffffffu, h16 ? v[k] : v[k + 4], 16);
#pragma unroll
  for (int k = 0; k < 2; ++k)
    u2[k] = (h8 ? u4[k + 2] : u4[k]) + __shfl_xor_sync(0xffffffffu, h8 ? u4[k] : u4[k + 2], 8);
  float u1 = (h4 ? u2[1] : u2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? u2[0] : u2[1], 4);
  u1 += __shfl_xor_sync(0xffffffffu, u1, 2);
  u1 += __shfl_xor_sync(0xffffffffu, u1, 1);
  return u1;
}

template <int MODE>
__global__ void __launch_bounds__(kTileThreads)
k_band_solve_tile(int N, int b, const float* __restrict__ tiles, const float* __restrict__ Dnb,
                  const float* __restrict__ vin, const double* __restrict__ dsq, float* __restrict__ ty,
                  float* __restrict__ tp, float* __restrict__ z, int ld, int c0, int ncols, int ring_mask,
                  int nst, int32_t* __restrict__ err) {
  constexpr bool kFwd = MODE <= FWD_P_FROM_V;
  constexpr int NB = kTileNB;
  constexpr int RB = NB / (kTileThreads / 32);  // tile rows per warp
  static_assert(RB == 4 && kCols == 2, "reduce8 sums 4 rows x 2 columns per warp");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // nst pipeline stages of (tile, block inverse); the ring holds every solution row twice,
  // slots j mod R and j mod R + R, R a power of two above the rows alive at once (W + NB)
  const int W = band_ld(b);
  const int R = ring_mask + 1;
  const size_t tbytes_al = align16((size_t)NB * W * sizeof(float));
  constexpr size_t dbytes_al = align16((size_t)NB * NB * sizeof(float));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // [nst], nst <= kTileMaxStages
  unsigned char* stage0 = smem_raw + 8 * kTileMaxStages;
  auto tdst = [&](int slot) { return reinterpret_cast<float*>(stage0 + slot * tbytes_al); };
  auto ddst = [&](int slot) { return reinterpret_cast<float*>(stage0 + nst * tbytes_al + slot * dbytes_al); };
  float* ring = reinterpret_cast<float*>(stage0 + nst * (tbytes_al + dbytes_al));  // [2R][kCols]
  float* tb = ring + (size_t)2 * R * kCols;                                               // [NB][kCols]
  const int cbase = c0 + blockIdx.x * kCols;
  const int ncl = min(kCols, c0 + ncols - cbase);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nblk = (N + NB - 1) / NB;
  const uint32_t tbytes = (uint32_t)((size_t)NB * W * sizeof(float));
  constexpr uint32_t dbytes = (uint32_t)(NB * NB * sizeof(float));
  // after the reductions lane `lane` holds row orow, column ocol (four lanes per output)
  const int oidx = (lane >> 2) & 7;
  const int orow = warp * RB + (oidx >> 1), ocol = oidx & 1;
  const bool owner = (lane & 3) == 0;

  auto read_rhs = [&](int i, int c) -> float {
    if (MODE == FWD_U_FROM_V) { const int rr = udof(i); return vin[(size_t)rr * ld + c] * (float)dsq[rr]; }
    if (MODE == FWD_P_FROM_T) return tp[(size_t)i * ld + c];
    if (MODE == FWD_P_FROM_V) { const int rr = 3 * i + 2; return -vin[(size_t)rr * ld + c] * (float)dsq[rr]; }
    if (MODE == BWD_U_TO_Z) return ty[(size_t)i * ld + c];
    return tp[(size_t)i * ld + c];
  };
  auto write_out = [&](int i, int c, float y) {
    if (MODE == FWD_U_FROM_V) ty[(size_t)i * ld + c] = y;
    else if (MODE == FWD_P_FROM_T || MODE == FWD_P_FROM_V) tp[(size_t)i * ld + c] = y;
    else if (MODE == BWD_U_TO_Z) z[(size_t)udof(i) * ld + c] = y;
    else z[(size_t)(3 * i + 2) * ld + c] = y;
  };
  auto block_of = [&](int bi) { return kFwd ? bi : (nblk - 1 - bi); };
  auto issue = [&](int bi, int sl) {
    const int I = block_of(bi);
    mbar_expect(&bar[sl], tbytes + dbytes);
    bulk_copy(tdst(sl), tiles + (size_t)I * NB * W, tbytes, &bar[sl]);
    bulk_copy(ddst(sl), Dnb + (size_t)I * NB * NB, dbytes, &bar[sl]);
  };

  // window rows that no block has written (j < 0, j >= N) meet zero tile entries: keep them finite
  for (int k = t; k < 2 * R * kCols; k += kTileThreads) ring[k] = 0.f;
  if (t == 0) {
    for (int k = 0; k < nst; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0)
    for (int k = 0; k < nst && k < nblk; ++k) issue(k, k);
  float rhs_next;
  {
    const int i = block_of(0) * NB + orow;
    rhs_next = (owner && ocol < ncl && i < N) ? read_rhs(i, cbase + ocol) : 0.f;
  }
  // stage and its barrier phase, and the window's first ring slot, advance with bi
  int slot = 0;
  uint32_t phase = 0;
  int s0 = (kFwd ? ((block_of(0) * NB - b) & ~1) : block_of(0) * NB + NB) & ring_mask;  // even
  for (int bi = 0; bi < nblk; ++bi) {
    const int I = block_of(bi);
    const int i0 = I * NB;
    const int io = i0 + orow;
    const float rhs = rhs_next;
    if (bi + 1 < nblk) {
      const int in = block_of(bi + 1) * NB + orow;
      rhs_next = (owner && ocol < ncl && in < N) ? read_rhs(in, cbase + ocol) : 0.f;
    }
    const bool ok = mbar_wait_bounded(&bar[slot], phase, c_first_wait_budget);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicExch(err, 1);
        // let copies still in flight land before the CTA's shared memory is released
        for (int k = bi; k < bi + nst && k < nblk; ++k)
          mbar_wait_bounded(&bar[k % nst], (uint32_t)((k / nst) & 1), kWaitBudget);
      }
      __syncthreads();
      return;
    }
    // off-block products: tile rows warp*RB .. warp*RB + RB - 1 times the solution window,
    // ring slots s0 .. s0 + W - 1 (s0 even, so the window's 16-byte chunks are aligned)
    const float* Trow = tdst(slot) + (size_t)(warp * RB) * W;
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
#pragma unroll 2
    for (int ch = lane; ch < W / 4; ch += 32) {
      const float4 ya = *reinterpret_cast<const float4*>(ring + (size_t)(s0 + 4 * ch) * kCols);
      const float4 yb = *reinterpret_cast<const float4*>(ring + (size_t)(s0 + 4 * ch + 2) * kCols);
#pragma unroll
      for (int rr = 0; rr < RB; ++rr) {
        const float4 tv = *reinterpret_cast<const float4*>(Trow + (size_t)rr * W + 4 * ch);
        float a0 = acc[2 * rr], a1 = acc[2 * rr + 1];
        a0 = fmaf(tv.x, ya.x, a0);
        a1 = fmaf(tv.x, ya.y, a1);
        a0 = fmaf(tv.y, ya.z, a0);
        a1 = fmaf(tv.y, ya.w, a1);
        a0 = fmaf(tv.z, yb.x, a0);
        a1 = fmaf(tv.z, yb.y, a1);
        a0 = fmaf(tv.w, yb.z, a0);
        a1 = fmaf(tv.w, yb.w, a1);
        acc[2 * rr] = a0;
        acc[2 * rr + 1] = a1;
      }
    }
    const float sum = reduce8(acc, lane);
    if (owner) tb[orow * kCols + ocol] = rhs - sum;
    __syncthreads();
    // diagonal block: y = D_I tb with D_I's NB x NB inverse (zero outside the triangle)
    {
      const float* D = ddst(slot);
      const int h = lane & 3;
      float y = 0.f;
      if (kFwd) {  // lower-triangular inverse: skip its exact zeros
        for (int k = h; k <= orow; k += 4) y = fmaf(D[orow * NB + k], tb[k * kCols + ocol], y);
      } else {
        for (int k = orow + ((h - orow) & 3); k < NB; k += 4) y = fmaf(D[k * NB + orow], tb[k * kCols + ocol], y);
      }
      y += __shfl_xor_sync(0xffffffffu, y, 1);
      y += __shfl_xor_sync(0xffffffffu, y, 2);
      if (owner && io < N) {
        const int sl = io & ring_mask;
        ring[(size_t)sl * kCols + ocol] = y;
        ring[(size_t)(sl + R) * kCols + ocol] = y;
        if (ocol < ncl) write_out(io, cbase + ocol, y);
      }
    }
    __syncthreads();
    // this stage is free again: prefetch block bi + nst into it
    if (t == 0 && bi + nst < nblk) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(bi + nst, slot);
    }
    if (++slot == nst) {
      slot = 0;
      phase ^= 1u;
    }
    s0 = (s0 + (kFwd ? NB : -NB)) & ring_mask;
  }
}

// Ring rows of the tile solve: a power of two above the W + NB rows alive at once.
int tile_ring_rows(int b) {
  int r = 2;
  while (r < band_ld(b) + kTileNB + 1) r <<= 1;
  return r;
}

// Shared memory of the tile solve with nst stages.
size_t tile_smem_bytes(int b, int nst) {
  return 8 * kTileMaxStages +
         nst * (align16((size_t)kTileNB * band_ld(b) * sizeof(float)) + align16((size_t)kTileNB * kTileNB * sizeof(float))) +
         2 * (size_t)tile_ring_rows(b) * kCols * sizeof(float) + (size_t)kTileNB * kCols * sizeof(float);
}

// As many bulk-copy stages as fit in 227 KB, at most kTileMaxStages (0 if fewer than 2 fit);
// a stage is refilled nst - 1 blocks before its use.
int tile_stages(int b) {
  for (int nst = kTileMaxStages; nst >= 2; --nst)
    if (tile_smem_bytes(b, nst) <= 227 * 1024) return nst;
  return 0;
}

template <int MODE>
static void launch_tile(biot_ctx* ctx, int N, int b, const float* tiles, const float* Dnb, const float* vin, float* z,
                        int c0, int ncols) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_band_solve_tile<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  const int nst = tile_stages(b);
  const size_t smem = tile_smem_bytes(b, nst);
  BIOT_LAUNCH(k_band_solve_tile<MODE>, div_up(ncols, kCols), kTileThreads, smem, ctx->stream, N, b, tiles, Dnb, vin,
              ctx->dsq, ctx->lp.tu, ctx->lp.tp, z, ctx->wcap, c0, ncols, tile_ring_rows(b) - 1, nst,
              ctx->status);
}

template <int MODE, typename T>
static void launch_legacy(biot_ctx* ctx, int N, int b, const T* band, const T* Dinv, const T* vin, T* z, int c0,
                          int ncols) {
  const int rr = ring_rows(b);
  const size_t smem = sizeof(T) * ((size_t)rr * kCols + kNB * kCols);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_band_solve<MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  BIOT_LAUNCH((k_band_solve<MODE, T>), div_up(ncols, kCols), kSolveThreads, smem, ctx->stream, N, b, band, Dinv, vin,
              ctx->dsc, BandBufs<T>::tu(ctx), BandBufs<T>::tp(ctx), z, ctx->wcap, c0, ncols, rr - 1);
}


// Band-solve variants the tuner chooses from: the register-streaming kernel, and
// TMA-staged kernels with NB-row blocks and THREADS threads.
const BandVariant kBandVariants[kBandVariantCount] = {
    {0, 64, 256}, {1, 16, 128}, {1, 16, 256}, {1, 32, 256}, {1, 8, 128}, {1, 32, 128}, {2, kTileNB, kTileThreads},
    {3, kRowsNB, 32}, {3, kRowsNB, 64}, {3, kRowsNB, 128}, {1, 4, 128}};

size_t band_variant_smem(int v, bool fp64, int b) {
  const BandVariant& V = kBandVariants[v];
  const size_t es = fp64 ? 8 : 4;
  if (!V.tma) return es * ((size_t)ring_rows(b) * kCols + kNB * kCols);
  if (V.tma == 2) return tile_stages(b) ? tile_smem_bytes(b, tile_stages(b)) : (size_t)1 << 30;
  return 64 + 2 * align16((size_t)V.nb * band_ld(b) * es) + 2 * align16((size_t)V.nb * V.nb * es) +
         2 * (size_t)tma_ring_rows(b, V.nb) * kCols * es + (size_t)V.nb * kCols * es;
}

bool band_variant_ok(int v, bool fp64, int b) {
  if (fp64 && kBandVariants[v].tma == 2) return false;  // the tile solve is FP32 only
  if (kBandVariants[v].tma == 3) return false;          // the row-per-lane solve is in-place only
  if (v == kWideVariant) return false;                  // so is the four-row TMA solve
  return band_variant_smem(v, fp64, b) <= 227 * 1024;
}

bool band_variant_inplace_ok(int v, bool fp64, int b) {
  if (kBandVariants[v].tma == 3) {
    const int w = kBandVariants[v].threads / 32;
    return (fp64 ? rows_smem_bytes<double>(b, w) : rows_smem_bytes<float>(b, w)) <= 227 * 1024;
  }
  return kBandVariants[v].tma == 1 && band_variant_smem(v, fp64, b) <= 227 * 1024;
}

int band_variant_default(bool fp64, int b) {
  const int pref = fp64 ? 2 : 6;  // TMA NB=16 x 256 threads (FP64), skewed tiles NB=32 x 256 threads (FP32)
  if (band_variant_ok(pref, fp64, b)) return pref;
  for (int v = kBandVariantCount - 1; v > 0; --v)
    if (band_variant_ok(v, fp64, b)) return v;
  return 0;
}


template <int MODE, typename T>
static void solve(biot_ctx* ctx, int variant, int N, int b, const T* band, const T* Dinv, const T* Dnb, const T* vin,
                  T* z, int c0, int ncols) {
  switch (variant) {
    case 1: launch_tma<MODE, T, 16, 128>(ctx, N, b, band, Dnb, vin, z, c0, ncols); break;
    case 2: launch_tma<MODE, T, 16, 256>(ctx, N, b, band, Dnb, vin, z, c0, ncols); break;
    case 3: launch_tma<MODE, T, 32, 256>(ctx, N, b, band, Dnb, vin, z, c0, ncols); break;
    case 4: launch_tma<MODE, T, 8, 128>(ctx, N, b, band, Dnb, vin, z, c0, ncols); break;
    case 5: launch_tma<MODE, T, 32, 128>(ctx, N, b, band, Dnb, vin, z, c0, ncols); break;
    case 6:
      if constexpr (sizeof(T) == 4) {
        constexpr bool u = MODE == FWD_U_FROM_V || MODE == BWD_U_TO_Z;
        constexpr bool fwd = MODE <= FWD_P_FROM_V;
        launch_tile<MODE>(ctx, N, b, ctx->lp.tile[u ? 0 : 1][fwd ? 0 : 1], Dnb, vin, z, c0, ncols);
      }
      break;
    default: launch_legacy<MODE, T>(ctx, N, b, band, Dinv, vin, z, c0, ncols); break;
  }
}

template <typename T>
static biot_status build_dnb(biot_ctx* ctx, bool u, int nb) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  void*& dst = u ? ctx->dnb_u[pi] : ctx->dnb_p[pi];
  int& have = u ? ctx->dnb_nb_u[pi] : ctx->dnb_nb_p[pi];
  if (have == nb) return BIOT_OK;
  const int N = u ? 2 * ctx->n_nodes : ctx->n_nodes;
  if (!dst) BIOT_TRY(dalloc(ctx, &dst, sizeof(T) * ((size_t)N + 64) * 32));
  const T* D64 = u ? BandBufs<T>::Du(ctx) : BandBufs<T>::Dp(ctx);
  BIOT_LAUNCH(k_extract_dnb<T>, 512, 256, 0, ctx->stream, D64, N, nb, (T*)dst);
  BIOT_CU(ctx, cudaGetLastError());
  have = nb;
  return BIOT_OK;
}

// Skewed block tiles of block u (A) or p (S), forward and backward, from the FP32 factors.
static biot_status ensure_tiles(biot_ctx* ctx, bool u) {
  const int k = u ? 0 : 1;
  if (ctx->lp.tile_ok[k]) return BIOT_OK;
  const int N = u ? 2 * ctx->n_nodes : ctx->n_nodes;
  const int b = u ? ctx->band_u : ctx->band_p;
  const size_t sz = (size_t)div_up(N, kTileNB) * kTileNB * band_ld(b);
  for (int d = 0; d < 2; ++d)
    if (!ctx->lp.tile[k][d]) BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.tile[k][d], sizeof(float) * sz));
  BIOT_LAUNCH(k_band_to_tiles, 1024, 256, 0, ctx->stream, u ? ctx->lp.Lu : ctx->lp.Lp, N, b, true, ctx->lp.tile[k][0]);
  BIOT_LAUNCH(k_band_to_tiles, 1024, 256, 0, ctx->stream, u ? ctx->lp.Uu : ctx->lp.Up, N, b, false, ctx->lp.tile[k][1]);
  BIOT_CU(ctx, cudaGetLastError());
  ctx->lp.tile_ok[k] = 1;
  return BIOT_OK;
}

biot_status ensure_dnb(biot_ctx* ctx, bool fp64, bool u, int variant) {
  if (!kBandVariants[variant].tma) return BIOT_OK;
  if (kBandVariants[variant].tma == 2 && !fp64) BIOT_TRY(ensure_tiles(ctx, u));
  return fp64 ? build_dnb<double>(ctx, u, kBandVariants[variant].nb)
              : build_dnb<float>(ctx, u, kBandVariants[variant].nb);
}


// Runs the launches of its scope on ctx->side instead of ctx->stream.
struct OnSide {
  biot_ctx* ctx;
  cudaStream_t keep;
  explicit OnSide(biot_ctx* c) : ctx(c), keep(c->stream) { ctx->stream = ctx->side; }
  ~OnSide() { ctx->stream = keep; }
};

// z = P^{-1} vin on columns [c0, c0 + ncols). The band-solve timing class brackets the
// whole apply (four solves, plus the coupling for P1) on the caller's stream.
template <typename T>
void precond_apply(biot_ctx* ctx, const T* vin, T* z, int c0, int ncols) {
  using B = BandBufs<T>;
  KTimer tm(ctx, BIOT_KC_BAND_SOLVE);
  if (ctx->gmg) {
    gmg_apply<T>(ctx, vin, z, c0, ncols);
    return;
  }
  const int nn = ctx->n_nodes;
  const int pi = sizeof(T) == 8 ? 0 : 1;
  const int vu = ctx->band_var_u[pi], vp = ctx->band_var_p[pi];
  auto solve_u = [&]() {
    if (ctx->sub[0]) {
      sub_apply<T>(ctx, 0, vin, z, c0, ncols);
      return;
    }
    solve<FWD_U_FROM_V, T>(ctx, vu, 2 * nn, ctx->band_u, B::Lu(ctx), B::Du(ctx), B::Dnbu(ctx), vin, z, c0, ncols);
    solve<BWD_U_TO_Z, T>(ctx, vu, 2 * nn, ctx->band_u, B::Uu(ctx), B::Du(ctx), B::Dnbu(ctx), vin, z, c0, ncols);
  };
  auto solve_p = [&](bool from_t) {
    if (ctx->sub[1]) {
      sub_apply<T>(ctx, 1, from_t ? nullptr : vin, z, c0, ncols);
      return;
    }
    if (from_t)
      solve<FWD_P_FROM_T, T>(ctx, vp, nn, ctx->band_p, B::Lp(ctx), B::Dp(ctx), B::Dnbp(ctx), vin, z, c0, ncols);
    else
      solve<FWD_P_FROM_V, T>(ctx, vp, nn, ctx->band_p, B::Lp(ctx), B::Dp(ctx), B::Dnbp(ctx), vin, z, c0, ncols);
    solve<BWD_P_TO_Z, T>(ctx, vp, nn, ctx->band_p, B::Up(ctx), B::Dp(ctx), B::Dnbp(ctx), vin, z, c0, ncols);
  };
  if (ctx->precond == BIOT_PRECOND_DIAG && ctx->side) {
    // P2 is block diagonal: A's solves (the long ones) on the high-priority side stream,
    // S's on the caller's stream, filling the SMs that A's CTAs leave free
    cudaEventRecord(ctx->ev_fork, ctx->stream);
    cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
    {
      OnSide on(ctx);
      solve_u();
    }
    solve_p(false);
    cudaEventRecord(ctx->ev_join, ctx->side);
    cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
    return;
  }
  solve_u();
  if (ctx->precond == BIOT_PRECOND_TRI) {
    launch_coupling<T>(ctx, z, vin, B::tp(ctx), c0, ncols);
    solve_p(true);
  } else {
    solve_p(false);
  }
}

// Time one forward + backward solve pair of block u (A) or p (S) with a variant.
template <typename T>
float time_band_pair(biot_ctx* ctx, bool u, int variant, const T* vin, T* z, int ncols) {
  using B = BandBufs<T>;
  const int nn = ctx->n_nodes;
  if (ensure_dnb(ctx, sizeof(T) == 8, u, variant) != BIOT_OK) return 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool was = ctx->timing;
  ctx->timing = false;
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, ctx->stream);
    if (u) {
      solve<FWD_U_FROM_V, T>(ctx, variant, 2 * nn, ctx->band_u, B::Lu(ctx), B::Du(ctx), B::Dnbu(ctx), vin, z, 0,
                             ncols);
      solve<BWD_U_TO_Z, T>(ctx, variant, 2 * nn, ctx->band_u, B::Uu(ctx), B::Du(ctx), B::Dnbu(ctx), vin, z, 0, ncols);
    } else {
      solve<FWD_P_FROM_V, T>(ctx, variant, nn, ctx->band_p, B::Lp(ctx), B::Dp(ctx), B::Dnbp(ctx), vin, z, 0, ncols);
      solve<BWD_P_TO_Z, T>(ctx, variant, nn, ctx->band_p, B::Up(ctx), B::Dp(ctx), B::Dnbp(ctx), vin, z, 0, ncols);
    }
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  ctx->timing = was;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

template float time_band_pair<double>(biot_ctx*, bool, int, const double*, double*, int);
template float time_band_pair<float>(biot_ctx*, bool, int, const float*, float*, int);

template void precond_apply<double>(biot_ctx*, const double*, double*, int, int);

size_t batched_solve_smem(int max_band) { return tma_smem_bytes<float, kBatchNB>(max_band); }

biot_status ensure_batch_dnb(biot_ctx* ctx) {
  if (ctx->lp.bdnb_ok) return BIOT_OK;
  for (int w = 0; w < 2; ++w) {
    const int N = w == 0 ? 2 * ctx->n_nodes : ctx->n_nodes;
    if (!ctx->lp.bdnb[w]) BIOT_TRY(dalloc(ctx, (void**)&ctx->lp.bdnb[w], sizeof(float) * ((size_t)N + 64) * 32));
    BIOT_LAUNCH(k_extract_dnb<float>, 512, 256, 0, ctx->stream, w == 0 ? ctx->lp.Du : ctx->lp.Dp, N, kBatchNB,
                ctx->lp.bdnb[w]);
  }
  BIOT_CU(ctx, cudaGetLastError());
  ctx->lp.bdnb_ok = 1;
  return BIOT_OK;
}

void batched_precond_apply(const InstDev* tab, int count, int j, int max_wcap, int max_band, bool tri,
                           cudaStream_t s) {
  const dim3 grid(div_up(max_wcap, kCols), 1, count);
  const size_t smem = batched_solve_smem(max_band);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(kb_band_solve_tma<FWD_U_FROM_V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(kb_band_solve_tma<BWD_U_TO_Z>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(kb_band_solve_tma<FWD_P_FROM_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(kb_band_solve_tma<FWD_P_FROM_V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(kb_band_solve_tma<BWD_P_TO_Z>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  BIOT_LAUNCH(kb_band_solve_tma<FWD_U_FROM_V>, grid, kBatchThreads, smem, s, tab, j);
  BIOT_LAUNCH(kb_band_solve_tma<BWD_U_TO_Z>, grid, kBatchThreads, smem, s, tab, j);
  if (tri) {
    launch_batched_coupling(tab, count, j, s);
    BIOT_LAUNCH(kb_band_solve_tma<FWD_P_FROM_T>, grid, kBatchThreads, smem, s, tab, j);
  } else {
    BIOT_LAUNCH(kb_band_solve_tma<FWD_P_FROM_V>, grid, kBatchThreads, smem, s, tab, j);
  }
  BIOT_LAUNCH(kb_band_solve_tma<BWD_P_TO_Z>, grid, kBatchThreads, smem, s, tab, j);
}
template void precond_apply<float>(biot_ctx*, const float*, float*, int, int);

// ---- building blocks of the substructured block solves ----

// Cholesky factor L of a band matrix (rows of Lb, zero beyond N), its transposed rows U and
// the inverses of its 64 x 64 diagonal blocks.
biot_status band_factor(biot_ctx* ctx, int N, int b, double* L, double* U, double* D) {
  BIOT_TRY(band_cholesky(ctx, N, b, L));
  BIOT_LAUNCH(k_band_transpose, div_up((long long)N * (b + 1), 256), 256, 0, ctx->stream, N, b, L, U);
  BIOT_LAUNCH(k_diag_inverse, div_up(N, kNB), 256, 0, ctx->stream, N, b, L, D);
  BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

// In-place forward (L y = buf) or backward (L^T x = buf) solve of columns [c0, c0 + ncols)
// of buf [rows][ld] with TMA variant `variant` (1..5). nstrips > 1: a block-diagonal band
// matrix of nstrips strips of N rows each (N a multiple of 64), solved strip-parallel.
template <typename T>
void band_solve_inplace(biot_ctx* ctx, bool fwd, int variant, int N, int nstrips, int b, const T* band,
                        const T* Dnb, T* buf, int ld, int c0, int ncols, int blk) {
#define BIOT_INPLACE_CASE(v, NB, TH)                                                                         \
  case v:                                                                                                    \
    if (fwd)                                                                                                 \
      launch_tma_raw<FWD_P_FROM_T, T, NB, TH>(ctx, N, b, band, Dnb, nullptr, nullptr, buf, nullptr, ld, c0,  \
                                              ncols, nstrips, N, blk);                                       \
    else                                                                                                     \
      launch_tma_raw<BWD_INPLACE, T, NB, TH>(ctx, N, b, band, Dnb, nullptr, nullptr, buf, nullptr, ld, c0,   \
                                             ncols, nstrips, N, blk);                                        \
    break;
  switch (variant) {
    case 7:
      if (fwd) launch_rows<FWD_P_FROM_T, T, 1>(ctx, N, b, band, Dnb, buf, ld, c0, ncols, nstrips);
      else launch_rows<BWD_INPLACE, T, 1>(ctx, N, b, band, Dnb, buf, ld, c0, ncols, nstrips);
      break;
    case 8:
      if (fwd) launch_rows<FWD_P_FROM_T, T, 2>(ctx, N, b, band, Dnb, buf, ld, c0, ncols, nstrips);
      else launch_rows<BWD_INPLACE, T, 2>(ctx, N, b, band, Dnb, buf, ld, c0, ncols, nstrips);
      break;
    case 9:
      if (fwd) launch_rows<FWD_P_FROM_T, T, 4>(ctx, N, b, band, Dnb, buf, ld, c0, ncols, nstrips);
      else launch_rows<BWD_INPLACE, T, 4>(ctx, N, b, band, Dnb, buf, ld, c0, ncols, nstrips);
      break;
    BIOT_INPLACE_CASE(1, 16, 128)
    BIOT_INPLACE_CASE(2, 16, 256)
    BIOT_INPLACE_CASE(3, 32, 256)
    BIOT_INPLACE_CASE(4, 8, 128)
    BIOT_INPLACE_CASE(5, 32, 128)
    BIOT_INPLACE_CASE(10, 4, 128)
    default: break;
  }
#undef BIOT_INPLACE_CASE
}
template void band_solve_inplace<double>(biot_ctx*, bool, int, int, int, int, const double*, const double*, double*,
                                         int, int, int, int);
template void band_solve_inplace<float>(biot_ctx*, bool, int, int, int, int, const float*, const float*, float*, int,
                                        int, int, int);

template <typename T>
void extract_dnb_raw(biot_ctx* ctx, const T* D64, int N, int nb, T* out) {
  BIOT_LAUNCH(k_extract_dnb<T>, 512, 256, 0, ctx->stream, D64, N, nb, out);
}
template void extract_dnb_raw<double>(biot_ctx*, const double*, int, int, double*);
template void extract_dnb_raw<float>(biot_ctx*, const float*, int, int, float*);

// The compact block inverses a variant reads (the row-per-lane solve: 16 x 16 at row stride 17).
template <typename T>
void extract_dnb_variant(biot_ctx* ctx, int variant, const T* D64, int N, T* out) {
  if (kBandVariants[variant].tma == 3) BIOT_LAUNCH(k_extract_dnb17<T>, 512, 256, 0, ctx->stream, D64, N, out);
  else extract_dnb_raw<T>(ctx, D64, N, kBandVariants[variant].nb, out);
}
template void extract_dnb_variant<double>(biot_ctx*, int, const double*, int, double*);
template void extract_dnb_variant<float>(biot_ctx*, int, const float*, int, float*);

void to_f32(biot_ctx* ctx, const double* in, float* out, size_t n) {
  BIOT_LAUNCH(k_to_f32, 1024, 256, 0, ctx->stream, in, out, n);
}

}  // namespace biot

extern "C" biot_status biot_debug_set_wait_budget(int64_t cycles) {
  const long long v = cycles <= 0 ? biot::kWaitBudget : std::min<long long>(cycles, biot::kWaitBudget);
  cudaError_t e = cudaMemcpyToSymbol(biot::c_first_wait_budget, &v, sizeof(v));
  if (e != cudaSuccess)
    return biot::fail(nullptr, BIOT_E_CUDA, "biot_debug_set_wait_budget: %s", cudaGetErrorString(e));
  return BIOT_OK;
}
