// Dense-block solves with the separators' Schur complement of the substructured blocks.
//
// Ssep (block tridiagonal: nsep = k - 1 separator lines of B = d (n + 1) DOFs) is factored by
// band Cholesky, Ssep = L L^T, with L block lower bidiagonal: dense lower-triangular diagonal
// blocks D_K and dense sub-diagonal blocks E_K = L[K][K-1]. The band substitution walks the
// nsep B rows a few at a time, a chain of nsep B / NB dependent steps on one SM per column
// pair. With the diagonal blocks' inverses formed once the same block substitution reads
//
//   forward  (L y = r):    z_K = D_K^{-1} r_K for all K at once,   y_0 = z_0,
//                          y_K = z_K - M_K y_{K-1},   M_K = D_K^{-1} E_K           (K = 1 ..)
//   backward (L^T x = y):  w_K = D_K^{-T} y_K for all K at once,   x_{nsep-1} = w_{nsep-1},
//                          x_K = w_K - P_K^T x_{K+1}, P_K = E_{K+1} D_K^{-1}       (K = .. 0)
//
// Per column the multiply-adds equal the substitution's (nsep B^2 / 2 for each block-diagonal
// product, (nsep - 1) B^2 for each chain), but the chain has nsep - 1 steps and each step is a
// dense B x B by B x ncols product spread over the whole GPU. D_K^{-1} is formed column by
// column by forward substitution on the unit vectors, M_K and P_K by the same product kernel.
// Errors grow with cond(D_K), the square root of the condition number of the diagonal block of
// Ssep's factorisation (an interface operator of the strip problems, far better conditioned
// than A itself).
#include "common.cuh"

#include <algorithm>

namespace biot {
namespace {

// E_K (K = 1 .. nsep - 1) as dense Bp x Bp blocks, E[(K - 1)][r][c] = L[K B + r][(K - 1) B + c],
// from Ssep's lower band (half-band bS = 2 B - 1: L[i][j] at band column bS - (i - j)).
__global__ void k_sep_extract_E(int nsep, int B, int Bp, int bS, const double* __restrict__ LS, int ldS,
                                double* __restrict__ E) {
  const long long tot = (long long)(nsep - 1) * B * B;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int K = 1 + (int)(t / ((long long)B * B));
    const int rc = (int)(t % ((long long)B * B)), r = rc / B, c = rc % B;
    const long long i = (long long)K * B + r, j = (long long)(K - 1) * B + c;
    E[(size_t)(K - 1) * Bp * Bp + (size_t)r * Bp + c] = LS[(size_t)i * ldS + (bS - (i - j))];
  }
}

// Column c of D_K^{-1} by forward substitution D_K x = e_c, one warp per column (four per
// CTA), x in shared memory: x_r = (delta_rc - sum_{c <= j < r} D_K[r][j] x_j) / D_K[r][r].
// Writes rows c .. B - 1 of column c (the rest of the zero-filled block stays zero).
constexpr int kInvWarps = 4;
__global__ void __launch_bounds__(kInvWarps * 32)
k_sep_inverse(int nsep, int B, int Bp, int bS, const double* __restrict__ LS, int ldS, double* __restrict__ Dinv) {
  extern __shared__ double xs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kInvWarps + warp, K = blockIdx.y;
  if (c >= B || K >= nsep) return;
  double* x = xs + (size_t)warp * B;
  double* out = Dinv + (size_t)K * Bp * Bp;
  for (int r = c; r < B; ++r) {
    // row r of D_K: D_K[r][j] = LS[(K B + r) ldS + bS - r + j]
    const double* Lr = LS + (size_t)((size_t)K * B + r) * ldS + (bS - r);
    double s = 0.0;
    for (int j = c + lane; j < r; j += 32) s = fma(Lr[j], x[j], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const double v = ((r == c ? 1.0 : 0.0) - s) / Lr[r];
    if (lane == 0) {
      x[r] = v;
      out[(size_t)r * Bp + c] = v;
    }
    __syncwarp();
  }
}

// C (=, -=) op(A) X on one B x B block: A is Bp x Bp row-major (zero beyond B), op(A) = A or
// A^T; X and C are B-row panels at row stride ld, columns [c0, c0 + ncols). blockIdx.z steps
// A, X and C by a_z, x_z and c_z elements (independent blocks of one batched product).
// TRI: A lower triangular, so op(A)'s tiles past the diagonal (right of it for A, left of it
// for A^T) are zero and skipped. BM x BM output tiles, 256 threads with (BM/16)^2 outputs
// each, 16-deep k tiles double-buffered through registers.
constexpr int kGemmBK = 16;

template <typename T, int BM, bool TRANS, bool SUB, bool TRI>
__global__ void __launch_bounds__(256)
k_sep_gemm(int B, int Bp, const T* __restrict__ A, long long a_z, const T* X, long long x_z, T* C, long long c_z,
           int ld, int c0, int ncols) {
  constexpr int BK = kGemmBK, TM = BM / 16, EA = BM * BK / 256;
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Xs[2][BK][BM];
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  // lower-triangular A: the last row tiles take the most k tiles, so they are issued first
  const int mt = (TRI && !TRANS) ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;
  const int n0 = blockIdx.x * BM, m0 = mt * BM;
  A += (size_t)blockIdx.z * a_z;
  X += (size_t)blockIdx.z * x_z;
  C += (size_t)blockIdx.z * c_z;
  int kbeg = 0, kend = Bp;
  if (TRI) {
    if (TRANS) kbeg = m0;                   // A^T upper: op(A)[m][k] = 0 for k < m
    else kend = min(Bp, m0 + BM);           // A lower:   op(A)[m][k] = 0 for k > m
  }
  T ra[EA], rx[EA];
  // tile loads: A (BM x BK of op(A)) and X (BK x BM), EA elements per thread
  auto load = [&](int k0) {
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      if (!TRANS) {
        const int mm = t / (BK / EA), kk = (t % (BK / EA)) * EA + e;
        ra[e] = A[(size_t)(m0 + mm) * Bp + k0 + kk];
      } else {
        const int kk = t / (BM / EA), mm = (t % (BM / EA)) * EA + e;
        ra[e] = A[(size_t)(k0 + kk) * Bp + m0 + mm];
      }
      const int kk = t / (BM / EA), nn = (t % (BM / EA)) * EA + e;
      const int k = k0 + kk, n = n0 + nn;
      rx[e] = (k < B && n < ncols) ? X[(size_t)k * ld + c0 + n] : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      if (!TRANS) {
        const int mm = t / (BK / EA), kk = (t % (BK / EA)) * EA + e;
        As[buf][kk][mm] = ra[e];
      } else {
        const int kk = t / (BM / EA), mm = (t % (BM / EA)) * EA + e;
        As[buf][kk][mm] = ra[e];
      }
      const int kk = t / (BM / EA), nn = (t % (BM / EA)) * EA + e;
      Xs[buf][kk][nn] = rx[e];
    }
  };
  T acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = T(0);
  int cur = 0;
  if (kbeg < kend) {
    load(kbeg);
    store(0);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], x[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[cur][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TM; ++j) x[j] = Xs[cur][kk][tx * TM + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    if (more) store(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty * TM + i;
    if (m >= B) continue;
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int n = n0 + tx * TM + j;
      if (n >= ncols) continue;
      T* cp = C + (size_t)m * ld + c0 + n;
      *cp = SUB ? *cp - acc[i][j] : acc[i][j];
    }
  }
}

// Which product: op(A) = A or A^T, C = or C -=, A lower triangular or full.
enum GemmKind { G_TRI = 0, G_TRI_T = 1, G_SUB = 2, G_SUB_T = 3, G_FULL = 4 };

template <typename T, int BM>
void gemm_bm(cudaStream_t st, GemmKind kind, dim3 grid, int B, int Bp, const T* A, long long a_z, const T* X,
             long long x_z, T* C, long long c_z, int ld, int c0, int ncols) {
  switch (kind) {
    case G_TRI:
      BIOT_LAUNCH((k_sep_gemm<T, BM, false, false, true>), grid, 256, 0, st, B, Bp, A, a_z, X, x_z, C, c_z, ld, c0, ncols);
      break;
    case G_TRI_T:
      BIOT_LAUNCH((k_sep_gemm<T, BM, true, false, true>), grid, 256, 0, st, B, Bp, A, a_z, X, x_z, C, c_z, ld, c0, ncols);
      break;
    case G_SUB:
      BIOT_LAUNCH((k_sep_gemm<T, BM, false, true, false>), grid, 256, 0, st, B, Bp, A, a_z, X, x_z, C, c_z, ld, c0, ncols);
      break;
    case G_SUB_T:
      BIOT_LAUNCH((k_sep_gemm<T, BM, true, true, false>), grid, 256, 0, st, B, Bp, A, a_z, X, x_z, C, c_z, ld, c0, ncols);
      break;
    default:
      BIOT_LAUNCH((k_sep_gemm<T, BM, false, false, false>), grid, 256, 0, st, B, Bp, A, a_z, X, x_z, C, c_z, ld, c0, ncols);
      break;
  }
}

// FP64: 32 x 32 tiles (the FP64 pipe, not shared memory, bounds even 2 x 2 outputs per thread,
// and the smaller tiles balance better). FP32: 64 x 64 tiles (half the shared-memory reads per
// multiply-add) when they give at least two CTAs per SM, 32 x 32 otherwise. Bp is a multiple of 64.
template <typename T>
void gemm(cudaStream_t st, GemmKind kind, int nz, int B, int Bp, const T* A, long long a_z, const T* X, long long x_z,
          T* C, long long c_z, int ld, int c0, int ncols) {
  if (nz < 1 || ncols < 1) return;
  const long long big = (long long)div_up(ncols, 64) * (Bp / 64) * nz;
  if (sizeof(T) == 4 && big >= 2 * 152) {
    gemm_bm<T, 64>(st, kind, dim3(div_up(ncols, 64), Bp / 64, nz), B, Bp, A, a_z, X, x_z, C, c_z, ld, c0, ncols);
  } else {
    gemm_bm<T, 32>(st, kind, dim3(div_up(ncols, 32), Bp / 32, nz), B, Bp, A, a_z, X, x_z, C, c_z, ld, c0, ncols);
  }
}

}  // namespace

biot_status sep_dense_setup(biot_ctx* ctx, SubBlock* sb) {
  const int nsep = sb->k - 1, B = sb->B, Bp = (B + 63) / 64 * 64;
  if (nsep < 1) return BIOT_OK;
  cudaStream_t st = ctx->stream;
  sb->Bp = Bp;
  const size_t blk = (size_t)Bp * Bp, nD = (size_t)nsep * blk, nM = (size_t)(nsep - 1) * blk;
  const int ldS = band_ld(sb->bS);
  BIOT_TRY(dalloc(ctx, (void**)&sb->Dinv, sizeof(double) * nD));
  BIOT_CU(ctx, cudaMemsetAsync(sb->Dinv, 0, sizeof(double) * nD, st));
  const size_t smem = sizeof(double) * kInvWarps * B;
  if (smem > 227 * 1024) return fail(ctx, BIOT_E_INVALID, "separator blocks of %d rows too large", B);
  if (smem > 48 * 1024)
    BIOT_CU(ctx, cudaFuncSetAttribute(k_sep_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BIOT_LAUNCH(k_sep_inverse, dim3(div_up(B, kInvWarps), nsep), kInvWarps * 32, smem, st, nsep, B, Bp, sb->bS, sb->LS,
              ldS, sb->Dinv);
  if (nsep > 1) {
    double* E = nullptr;
    BIOT_TRY(dalloc(ctx, (void**)&E, sizeof(double) * nM));
    BIOT_TRY(dalloc(ctx, (void**)&sb->Mk, sizeof(double) * nM));
    BIOT_TRY(dalloc(ctx, (void**)&sb->Pk, sizeof(double) * nM));
    BIOT_CU(ctx, cudaMemsetAsync(E, 0, sizeof(double) * nM, st));
    BIOT_CU(ctx, cudaMemsetAsync(sb->Mk, 0, sizeof(double) * nM, st));
    BIOT_CU(ctx, cudaMemsetAsync(sb->Pk, 0, sizeof(double) * nM, st));
    BIOT_LAUNCH(k_sep_extract_E, std::min(div_up((long long)(nsep - 1) * B * B, 256), 152 * 16), 256, 0, st, nsep, B,
                Bp, sb->bS, sb->LS, ldS, E);
    // M_K = D_K^{-1} E_K (K = 1 ..): stored at K - 1; P_K = E_{K+1} D_K^{-1} (K = 0 .. nsep - 2)
    gemm<double>(st, G_TRI, nsep - 1, B, Bp, sb->Dinv + blk, (long long)blk, E, (long long)blk, sb->Mk,
                 (long long)blk, Bp, 0, B);
    gemm<double>(st, G_FULL, nsep - 1, B, Bp, E, (long long)blk, sb->Dinv, (long long)blk, sb->Pk, (long long)blk, Bp,
                 0, B);
    BIOT_CU(ctx, cudaStreamSynchronize(st));
    dfree(ctx, E);
  }
  if (ctx->prm.precision != BIOT_FP64) {
    BIOT_TRY(dalloc(ctx, (void**)&sb->Dinvf, sizeof(float) * nD));
    to_f32(ctx, sb->Dinv, sb->Dinvf, nD);
    if (nsep > 1) {
      BIOT_TRY(dalloc(ctx, (void**)&sb->Mkf, sizeof(float) * nM));
      BIOT_TRY(dalloc(ctx, (void**)&sb->Pkf, sizeof(float) * nM));
      to_f32(ctx, sb->Mk, sb->Mkf, nM);
      to_f32(ctx, sb->Pk, sb->Pkf, nM);
    }
  }
  BIOT_CU(ctx, cudaGetLastError());
  sb->dense = true;
  return BIOT_OK;
}

// In place on tS (NS rows at stride ld, columns [c0, c0 + ncols)): tS = Ssep^{-1} tS, with tZ
// (same shape) as the forward result.
template <typename T>
void sep_dense_solve(biot_ctx* ctx, SubBlock* sb, T* tS, T* tZ, int ld, int c0, int ncols) {
  const int nsep = sb->k - 1, B = sb->B, Bp = sb->Bp;
  const long long blk = (long long)Bp * Bp, rows = (long long)B * ld;
  const bool f = sizeof(T) == 4;
  const T* Dinv = f ? (const T*)sb->Dinvf : (const T*)sb->Dinv;
  const T* Mk = f ? (const T*)sb->Mkf : (const T*)sb->Mk;
  const T* Pk = f ? (const T*)sb->Pkf : (const T*)sb->Pk;
  cudaStream_t st = ctx->stream;
  // forward: z = blockdiag(D^{-1}) r, then y_K = z_K - M_K y_{K-1}
  gemm<T>(st, G_TRI, nsep, B, Bp, Dinv, blk, tS, rows, tZ, rows, ld, c0, ncols);
  for (int K = 1; K < nsep; ++K)
    gemm<T>(st, G_SUB, 1, B, Bp, Mk + (size_t)(K - 1) * blk, 0, tZ + (size_t)(K - 1) * rows, 0,
            tZ + (size_t)K * rows, 0, ld, c0, ncols);
  // backward: w = blockdiag(D^{-T}) y, then x_K = w_K - P_K^T x_{K+1}
  gemm<T>(st, G_TRI_T, nsep, B, Bp, Dinv, blk, tZ, rows, tS, rows, ld, c0, ncols);
  for (int K = nsep - 2; K >= 0; --K)
    gemm<T>(st, G_SUB_T, 1, B, Bp, Pk + (size_t)K * blk, 0, tS + (size_t)(K + 1) * rows, 0, tS + (size_t)K * rows, 0,
            ld, c0, ncols);
}
template void sep_dense_solve<double>(biot_ctx*, SubBlock*, double*, double*, int, int, int);
template void sep_dense_solve<float>(biot_ctx*, SubBlock*, float*, float*, int, int, int);

}  // namespace biot
