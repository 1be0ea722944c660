// The inner solver K(P, AA, X, b, n_iter) of Algorithm 3, batched over the
// active time steps of a sweep.
//
// One cycle of right-preconditioned flexible GMRES per step (the paper uses
// PETSc GMRES, Sec. 4; the preconditioner apply is exact here, the flexible
// form keeps Z = P^{-1} V explicitly for the update). The Arnoldi basis lives in
// the equilibrated variables r~ = D^{-1/2} r, D = |diag AA|, so the minimised
// norm weighs the displacement and pressure equations alike:
//   v_0 = r~ / |r~|;  z_j = P^{-1} (D^{1/2} v_j);  w = D^{-1/2} AA z_j;
//   classical Gram-Schmidt applied twice; Givens rotations on H;
//   x <- x + Z_k y_k with R y = g.
// Every reduction (dot products, norms) is a fixed two-level tree: per-block
// partial sums, then a pass over the blocks in order. Results do not depend on
// scheduling.
#include "common.cuh"

#include <algorithm>

namespace biot {

namespace {

constexpr int kRecH = (kMaxIter + 1) * kMaxIter;              // H, row-major (kMaxIter+1) x kMaxIter
constexpr int kRecG = kRecH;                                  // g[kMaxIter+1]
constexpr int kRecCS = kRecG + kMaxIter + 1;                  // cs[kMaxIter]
constexpr int kRecSN = kRecCS + kMaxIter;                     // sn[kMaxIter]
constexpr int kRecY = kRecSN + kMaxIter;                      // y[kMaxIter]
constexpr int kRec = kRecY + kMaxIter;

// out[s][c] = sum over blocks of part[s][block][c], s < nslots, c in [c0, c0 + ncols).
__device__ __forceinline__ void reduce_body(const double* __restrict__ part, int nblocks, int nslots, int ld, int c0,
                                            int ncols, double* __restrict__ out, int ldo) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (c >= c0 + ncols || s >= nslots) return;
  double acc = 0.0;
  const double* p = part + (size_t)s * nblocks * ld + c;
  for (int b = 0; b < nblocks; ++b) acc += p[(size_t)b * ld];
  out[(size_t)s * ldo + c] = acc;
}

// The same sums with one warp per column: lane l adds blocks l, l + 32, l + 64, ... in order,
// then the 32 lane sums are combined by a fixed butterfly (a fixed tree: deterministic).
// Block: 8 warps = 8 columns.
__global__ void __launch_bounds__(256) k_reduce_warp(const double* __restrict__ part, int nblocks, int nslots, int ld,
                                                     int c0, int ncols, double* __restrict__ out, int ldo) {
  const int lane = threadIdx.x & 31;
  const int cc = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int s = blockIdx.y;
  if (cc >= ncols) return;  // whole warps leave together
  const int c = c0 + cc;
  const double* p = part + (size_t)s * nblocks * ld + c;
  double acc = 0.0;
  for (int b = lane; b < nblocks; b += 32) acc += p[(size_t)b * ld];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[(size_t)s * ldo + c] = acc;
}

// Partial dot products part[i][block][c] = sum_{rows of block} V_i[r][c] * w[r][c]
// (products accumulated in T within a thread, combined in FP64 across threads and blocks).
template <typename T>
__device__ __forceinline__ void dots_body(const T* __restrict__ V, size_t vstride, const T* __restrict__ w, int nrows,
                                          int ld, int c0, int ncols, double* __restrict__ part) {
  __shared__ double sm[8][32];
  const int i = blockIdx.y;
  const T* Vi = V + (size_t)i * vstride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nrows + gridDim.x - 1) / gridDim.x;
  const int rb = blockIdx.x * per, re = min(nrows, rb + per);
  for (int cb = 0; cb < ncols; cb += 32) {
    const int c = c0 + cb + lane;
    const bool cv = cb + lane < ncols;
    T acc = 0;
    if (cv)
      for (int r = rb + warp; r < re; r += 8) acc += Vi[(size_t)r * ld + c] * w[(size_t)r * ld + c];
    sm[warp][lane] = (double)acc;
    __syncthreads();
    if (warp == 0 && cv) {
      double s = 0.0;
      for (int k = 0; k < 8; ++k) s += sm[k][lane];
      part[((size_t)i * gridDim.x + blockIdx.x) * ld + c] = s;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_dots(const T* __restrict__ V, size_t vstride, const T* __restrict__ w, int nrows, int ld, int c0, int ncols,
       double* __restrict__ part) {
  dots_body<T>(V, vstride, w, nrows, ld, c0, ncols, part);
}

// 16-byte vectors of T (four floats or two doubles).
template <typename T> struct KVec;
template <> struct KVec<float> {
  using V = float4;
  static constexpr int n = 4;
  __device__ __forceinline__ static void get(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ __forceinline__ static V make(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <> struct KVec<double> {
  using V = double2;
  static constexpr int n = 2;
  __device__ __forceinline__ static void get(const V& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ __forceinline__ static V make(const double* o) { return make_double2(o[0], o[1]); }
};

// dots_body for nvec vectors in one pass: w is read once per chunk of kDotChunk vectors and
// every access is a 16-byte vector (a lane owns VEC consecutive columns; the column range is
// widened down to a multiple of VEC). Each column's products are summed in the same order as
// in dots_body, so the partials are identical. Needs ld % VEC == 0 and 16-byte aligned rows.
constexpr int kDotChunk = 8;
constexpr int kFuseVecs = 12;  // basis vectors up to which the first update also forms the second's dots
template <typename T>
__global__ void __launch_bounds__(256, 3)
k_dots_vec(const T* __restrict__ V, size_t vstride, int nvec, const T* __restrict__ w, int nrows, int ld, int c0,
           int ncols, double* __restrict__ part) {
  using VV = typename KVec<T>::V;
  constexpr int VEC = KVec<T>::n;
  __shared__ double sm[8][32 * VEC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nrows + gridDim.x - 1) / gridDim.x;
  const int rb = blockIdx.x * per, re = min(nrows, rb + per);
  const int ca = c0 & ~(VEC - 1), ce = c0 + ncols;
  for (int cb = ca; cb < ce; cb += 32 * VEC) {
    const int c = cb + lane * VEC;
    const bool any = c < ce;
    for (int i0 = 0; i0 < nvec; i0 += kDotChunk) {
      const int ni = min(kDotChunk, nvec - i0);
      T acc[kDotChunk][VEC];
#pragma unroll
      for (int ii = 0; ii < kDotChunk; ++ii)
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[ii][q] = T(0);
      if (any) {
        for (int r = rb + warp; r < re; r += 8) {
          T wv[VEC];
          KVec<T>::get(*reinterpret_cast<const VV*>(w + (size_t)r * ld + c), wv);
#pragma unroll
          for (int ii = 0; ii < kDotChunk; ++ii) {
            if (ii < ni) {
              T v[VEC];
              KVec<T>::get(*reinterpret_cast<const VV*>(V + (size_t)(i0 + ii) * vstride + (size_t)r * ld + c), v);
#pragma unroll
              for (int q = 0; q < VEC; ++q) acc[ii][q] += v[q] * wv[q];
            }
          }
        }
      }
      for (int ii = 0; ii < ni; ++ii) {
        // the compiler keeps acc in registers: ii is a runtime index only in this epilogue
#pragma unroll
        for (int k = 0; k < kDotChunk; ++k)
          if (k == ii)
#pragma unroll
            for (int q = 0; q < VEC; ++q) sm[warp][lane * VEC + q] = (double)acc[k][q];
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * VEC; t += blockDim.x) {
          const int col = cb + t;
          if (col >= c0 && col < ce) {
            double sum = 0.0;
            for (int u = 0; u < 8; ++u) sum += sm[u][t];
            part[((size_t)(i0 + ii) * gridDim.x + blockIdx.x) * ld + col] = sum;
          }
        }
        __syncthreads();
      }
    }
  }
}

// w -= V h on the columns [c0, c0 + ncols) with the blocks owning row ranges (warps stride
// the rows, a lane owns VEC consecutive columns, so every row access is one coalesced 16-byte
// vector per lane) and the coefficients h[i][c] staged in shared memory per 32 VEC columns.
// Same per-element arithmetic order as gs_axpy_body. NORM: also the per-block partial sums
// of |w|^2 after the update, in part[block][c] (the layout k_dots_vec writes for one vector),
// which saves the separate norm pass of the second Gram-Schmidt sweep.
template <typename T, bool NORM>
__global__ void __launch_bounds__(256)
k_gs_axpy_rows_vec(const T* __restrict__ V, size_t vstride, int nvec, const double* __restrict__ h,
                   T* __restrict__ w, int nrows, int ld, int c0, int ncols, double* __restrict__ part) {
  using VV = typename KVec<T>::V;
  constexpr int VEC = KVec<T>::n;
  __shared__ __align__(16) T sh[kMaxIter + 1][32 * VEC];
  __shared__ double sm[NORM ? 8 : 1][NORM ? 32 * VEC : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nrows + gridDim.x - 1) / gridDim.x;
  const int rb = blockIdx.x * per, re = min(nrows, rb + per);
  const int ca = c0 & ~(VEC - 1), ce = c0 + ncols;
  for (int cb = ca; cb < ce; cb += 32 * VEC) {
    __syncthreads();
    for (int t = threadIdx.x; t < nvec * 32 * VEC; t += blockDim.x) {
      const int i = t / (32 * VEC), q = t % (32 * VEC), col = cb + q;
      sh[i][q] = col < ld ? (T)h[(size_t)i * ld + col] : T(0);
    }
    __syncthreads();
    const int c = cb + lane * VEC;
    const bool any = c < ce;
    const bool full = c >= c0 && c + VEC <= ce;
    T nrm[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) nrm[q] = T(0);
    if (any) {
      for (int r = rb + warp; r < re; r += 8) {
        T* wr = w + (size_t)r * ld + c;
        T acc[VEC];
        KVec<T>::get(*reinterpret_cast<const VV*>(wr), acc);
#pragma unroll 4
        for (int i = 0; i < nvec; ++i) {
          T v[VEC], hq[VEC];
          KVec<T>::get(*reinterpret_cast<const VV*>(V + (size_t)i * vstride + (size_t)r * ld + c), v);
          KVec<T>::get(*reinterpret_cast<const VV*>(&sh[i][lane * VEC]), hq);
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[q] -= hq[q] * v[q];
        }
        if (full) {
          *reinterpret_cast<VV*>(wr) = KVec<T>::make(acc);
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q)
            if (c + q >= c0 && c + q < ce) wr[q] = acc[q];
        }
        if (NORM)
#pragma unroll
          for (int q = 0; q < VEC; ++q)
            if (c + q >= c0 && c + q < ce) nrm[q] += acc[q] * acc[q];
      }
    }
    if (NORM) {
#pragma unroll
      for (int q = 0; q < VEC; ++q) sm[warp][lane * VEC + q] = (double)nrm[q];
      __syncthreads();
      for (int t = threadIdx.x; t < 32 * VEC; t += blockDim.x) {
        const int col = cb + t;
        if (col >= c0 && col < ce) {
          double sum = 0.0;
          for (int u = 0; u < 8; ++u) sum += sm[u][t];
          part[(size_t)blockIdx.x * ld + col] = sum;
        }
      }
    }
  }
}

// The first Gram-Schmidt sweep fused with the dot products of the second: w -= V h (h the
// first sweep's coefficients, staged in shared memory as in k_gs_axpy_rows_vec; same
// per-element arithmetic order), then the per-block partials of V_i . w with the updated w
// as stored, in part[i][block][c]. The row partition, each thread's row order and the block
// epilogue are k_dots_vec's, so on the same grid the partials are bit-identical to a separate
// k_dots_vec pass over the stored w: one pass over V instead of two. V_i's row is read again for
// the dot after the update (from L1/L2: the same 16 bytes the update just loaded). Needs
// nvec <= NV: the dot accumulators live in registers, which leave room for two CTAs per SM, so
// it runs on 2 x 152 CTAs (k_dots_vec on 3 x 152); 8-byte vectors on 3 x 152 measured 13 %
// slower.
template <typename T, int NV>
__global__ void __launch_bounds__(256, 2)
k_gs_axpy_dots_vec(const T* __restrict__ V, size_t vstride, int nvec, const double* __restrict__ h,
                   T* __restrict__ w, int nrows, int ld, int c0, int ncols, double* __restrict__ part) {
  using KV = KVec<T>;
  using VV = typename KV::V;
  constexpr int VEC = KV::n;
  __shared__ __align__(16) T sh[NV][32 * VEC];
  __shared__ double sm[8][32 * VEC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nrows + gridDim.x - 1) / gridDim.x;
  const int rb = blockIdx.x * per, re = min(nrows, rb + per);
  const int ca = c0 & ~(VEC - 1), ce = c0 + ncols;
  for (int cb = ca; cb < ce; cb += 32 * VEC) {
    __syncthreads();
    for (int t = threadIdx.x; t < nvec * 32 * VEC; t += blockDim.x) {
      const int i = t / (32 * VEC), q = t % (32 * VEC), col = cb + q;
      sh[i][q] = col < ld ? (T)h[(size_t)i * ld + col] : T(0);
    }
    __syncthreads();
    const int c = cb + lane * VEC;
    const bool any = c < ce;
    const bool full = c >= c0 && c + VEC <= ce;
    T dacc[NV][VEC];
#pragma unroll
    for (int ii = 0; ii < NV; ++ii)
#pragma unroll
      for (int q = 0; q < VEC; ++q) dacc[ii][q] = T(0);
    if (any) {
      for (int r = rb + warp; r < re; r += 8) {
        T* wr = w + (size_t)r * ld + c;
        T acc[VEC];
        KV::get(*reinterpret_cast<const VV*>(wr), acc);
#pragma unroll 4
        for (int i = 0; i < nvec; ++i) {
          T v[VEC], hq[VEC];
          KV::get(*reinterpret_cast<const VV*>(V + (size_t)i * vstride + (size_t)r * ld + c), v);
          KV::get(*reinterpret_cast<const VV*>(&sh[i][lane * VEC]), hq);
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[q] -= hq[q] * v[q];
        }
        if (full) {
          *reinterpret_cast<VV*>(wr) = KV::make(acc);
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q)
            if (c + q >= c0 && c + q < ce) wr[q] = acc[q];
        }
#pragma unroll
        for (int ii = 0; ii < NV; ++ii) {
          if (ii < nvec) {
            T v[VEC];
            KV::get(*reinterpret_cast<const VV*>(V + (size_t)ii * vstride + (size_t)r * ld + c), v);
#pragma unroll
            for (int q = 0; q < VEC; ++q) dacc[ii][q] += v[q] * acc[q];
          }
        }
      }
    }
    for (int ii = 0; ii < nvec; ++ii) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k == ii)
#pragma unroll
          for (int q = 0; q < VEC; ++q) sm[warp][lane * VEC + q] = (double)dacc[k][q];
      __syncthreads();
      for (int t = threadIdx.x; t < 32 * VEC; t += blockDim.x) {
        const int col = cb + t;
        if (col >= c0 && col < ce) {
          double sum = 0.0;
          for (int u = 0; u < 8; ++u) sum += sm[u][t];
          part[((size_t)ii * gridDim.x + blockIdx.x) * ld + col] = sum;
        }
      }
      __syncthreads();
    }
  }
}

// k_gs_axpy_dots_vec for up to kDotChunk basis vectors with the dot accumulators in shared
// memory (each thread owns its slots; the per-column order of the sums is unchanged), which
// frees the registers for three CTAs per SM: it runs on k_dots_vec's grid (3 x 152 CTAs), so its
// partials are bit-identical to a k_dots_vec pass over the stored w.
template <typename T>
__global__ void __launch_bounds__(256, 3)
k_gs_axpy_dots_smem(const T* __restrict__ V, size_t vstride, int nvec, const double* __restrict__ h,
                    T* __restrict__ w, int nrows, int ld, int c0, int ncols, double* __restrict__ part) {
  using KV = KVec<T>;
  using VV = typename KV::V;
  constexpr int VEC = KV::n;
  constexpr int NV = kDotChunk;
  __shared__ __align__(16) T sh[NV][32 * VEC];
  __shared__ __align__(16) T dsm[8][NV][32 * VEC];
  __shared__ double sm[8][32 * VEC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nrows + gridDim.x - 1) / gridDim.x;
  const int rb = blockIdx.x * per, re = min(nrows, rb + per);
  const int ca = c0 & ~(VEC - 1), ce = c0 + ncols;
  for (int cb = ca; cb < ce; cb += 32 * VEC) {
    __syncthreads();
    for (int t = threadIdx.x; t < nvec * 32 * VEC; t += blockDim.x) {
      const int i = t / (32 * VEC), q = t % (32 * VEC), col = cb + q;
      sh[i][q] = col < ld ? (T)h[(size_t)i * ld + col] : T(0);
    }
    T zero[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) zero[q] = T(0);
    for (int ii = 0; ii < nvec; ++ii) *reinterpret_cast<VV*>(&dsm[warp][ii][lane * VEC]) = KV::make(zero);
    __syncthreads();
    const int c = cb + lane * VEC;
    const bool any = c < ce;
    const bool full = c >= c0 && c + VEC <= ce;
    if (any) {
      for (int r = rb + warp; r < re; r += 8) {
        T* wr = w + (size_t)r * ld + c;
        T acc[VEC];
        KV::get(*reinterpret_cast<const VV*>(wr), acc);
#pragma unroll 4
        for (int i = 0; i < nvec; ++i) {
          T v[VEC], hq[VEC];
          KV::get(*reinterpret_cast<const VV*>(V + (size_t)i * vstride + (size_t)r * ld + c), v);
          KV::get(*reinterpret_cast<const VV*>(&sh[i][lane * VEC]), hq);
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[q] -= hq[q] * v[q];
        }
        if (full) {
          *reinterpret_cast<VV*>(wr) = KV::make(acc);
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q)
            if (c + q >= c0 && c + q < ce) wr[q] = acc[q];
        }
#pragma unroll 2
        for (int ii = 0; ii < nvec; ++ii) {
          T v[VEC], d[VEC];
          KV::get(*reinterpret_cast<const VV*>(V + (size_t)ii * vstride + (size_t)r * ld + c), v);
          VV* slot = reinterpret_cast<VV*>(&dsm[warp][ii][lane * VEC]);
          KV::get(*slot, d);
#pragma unroll
          for (int q = 0; q < VEC; ++q) d[q] += v[q] * acc[q];
          *slot = KV::make(d);
        }
      }
    }
    for (int ii = 0; ii < nvec; ++ii) {
#pragma unroll
      for (int q = 0; q < VEC; ++q) sm[warp][lane * VEC + q] = (double)dsm[warp][ii][lane * VEC + q];
      __syncthreads();
      for (int t = threadIdx.x; t < 32 * VEC; t += blockDim.x) {
        const int col = cb + t;
        if (col >= c0 && col < ce) {
          double sum = 0.0;
          for (int u = 0; u < 8; ++u) sum += sm[u][t];
          part[((size_t)ii * gridDim.x + blockIdx.x) * ld + col] = sum;
        }
      }
      __syncthreads();
    }
  }
}

// scale_cols_body with 16-byte accesses (src may alias dst).
template <typename T>
__global__ void k_scale_cols_vec(const T* src, T* dst, const double* __restrict__ scale, int nrows, int ld, int c0,
                                 int ncols) {
  using VV = typename KVec<T>::V;
  constexpr int VEC = KVec<T>::n;
  const int ca = c0 & ~(VEC - 1), ce = c0 + ncols;
  const int ngrp = (ce - ca + VEC - 1) / VEC;
  const long long total = (long long)nrows * ngrp;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ngrp), c = ca + (int)(idx % ngrp) * VEC;
    T v[VEC];
    KVec<T>::get(*reinterpret_cast<const VV*>(src + (size_t)r * ld + c), v);
#pragma unroll
    for (int q = 0; q < VEC; ++q) v[q] = v[q] * (T)scale[c + q];
    T* d = dst + (size_t)r * ld + c;
    if (c >= c0 && c + VEC <= ce) {
      *reinterpret_cast<VV*>(d) = KVec<T>::make(v);
    } else {
#pragma unroll
      for (int q = 0; q < VEC; ++q)
        if (c + q >= c0 && c + q < ce) d[q] = v[q];
    }
  }
}

// w[r][c] -= sum_i h[i][c] V_i[r][c] (grid-stride over (r, c)).
template <typename T>
__device__ __forceinline__ void gs_axpy_body(const T* __restrict__ V, size_t vstride, int nvec,
                                             const double* __restrict__ h, T* __restrict__ w, int nrows, int ld,
                                             int c0, int ncols) {
  const long long total = (long long)nrows * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    T acc = w[(size_t)r * ld + c];
    for (int i = 0; i < nvec; ++i) acc -= (T)h[(size_t)i * ld + c] * V[(size_t)i * vstride + (size_t)r * ld + c];
    w[(size_t)r * ld + c] = acc;
  }
}

template <typename T>
__global__ void k_gs_axpy(const T* __restrict__ V, size_t vstride, int nvec, const double* __restrict__ h,
                          T* __restrict__ w, int nrows, int ld, int c0, int ncols) {
  gs_axpy_body<T>(V, vstride, nvec, h, w, nrows, ld, c0, ncols);
}

// dst[r][c] = src[r][c] * scale[c] (grid-stride).
template <typename T>
__device__ __forceinline__ void scale_cols_body(const T* src, T* dst,  // may alias (in-place scaling)
                                                const double* __restrict__ scale, int nrows, int ld, int c0,
                                                int ncols) {
  const long long total = (long long)nrows * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    dst[(size_t)r * ld + c] = src[(size_t)r * ld + c] * (T)scale[c];
  }
}

template <typename T>
__global__ void k_scale_cols(const T* src, T* dst, const double* __restrict__ scale,
                             int nrows, int ld, int c0, int ncols) {
  scale_cols_body<T>(src, dst, scale, nrows, ld, c0, ncols);
}

__device__ __forceinline__ void fgmres_init_body(double* __restrict__ cs, int ld, int c0, int ncols,
                                                 double* __restrict__ rec, int32_t* __restrict__ kcol) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c0 + ncols) return;
  const double beta0 = sqrt(cs[CS_RR * ld + c]);
  double* R = rec + (size_t)c * kRec;
  for (int k = 0; k < kRec; ++k) R[k] = 0.0;
  R[kRecG] = beta0;
  cs[CS_BETA0 * ld + c] = beta0;
  const bool act = beta0 > 0.0;
  cs[CS_ACTIVE * ld + c] = act ? 1.0 : 0.0;
  cs[CS_INVH * ld + c] = act ? 1.0 / beta0 : 0.0;
  kcol[c] = 0;
}

__global__ void k_fgmres_init(double* __restrict__ cs, int ld, int c0, int ncols, double* __restrict__ rec,
                              int32_t* __restrict__ kcol) {
  fgmres_init_body(cs, ld, c0, ncols, rec, kcol);
}

// Arnoldi step j of column c: store H[:, j], rotate, extend g, test breakdown.
__device__ __forceinline__ void givens_body(int j, double* __restrict__ cs, const double* __restrict__ h1,
                                            const double* __restrict__ h2, int ld, int c0, int ncols,
                                            double* __restrict__ rec, int32_t* __restrict__ kcol) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c0 + ncols) return;
  if (cs[CS_ACTIVE * ld + c] == 0.0) {
    cs[CS_INVH * ld + c] = 0.0;
    return;
  }
  double* R = rec + (size_t)c * kRec;
  double* H = R;
  double* g = R + kRecG;
  double* cc = R + kRecCS;
  double* sn = R + kRecSN;
  for (int i = 0; i <= j; ++i) H[i * kMaxIter + j] = h1[(size_t)i * ld + c] + h2[(size_t)i * ld + c];
  const double hn = sqrt(cs[CS_WW * ld + c]);
  const double wn0 = sqrt(cs[CS_WN0 * ld + c]);
  H[(j + 1) * kMaxIter + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * kMaxIter + j], b = H[(i + 1) * kMaxIter + j];
    H[i * kMaxIter + j] = cc[i] * a + sn[i] * b;
    H[(i + 1) * kMaxIter + j] = -sn[i] * a + cc[i] * b;
  }
  const double a = H[j * kMaxIter + j], b = H[(j + 1) * kMaxIter + j];
  const double den = hypot(a, b);
  if (den == 0.0) {
    cc[j] = 1.0;
    sn[j] = 0.0;
  } else {
    cc[j] = a / den;
    sn[j] = b / den;
  }
  H[j * kMaxIter + j] = den;
  H[(j + 1) * kMaxIter + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cc[j] * g[j];
  kcol[c] = j + 1;
  if (hn <= kBreakdownRtol * wn0) {
    cs[CS_ACTIVE * ld + c] = 0.0;
    cs[CS_INVH * ld + c] = 0.0;
  } else {
    cs[CS_INVH * ld + c] = 1.0 / hn;
  }
}

__global__ void k_givens(int j, double* __restrict__ cs, const double* __restrict__ h1, const double* __restrict__ h2,
                         int ld, int c0, int ncols, double* __restrict__ rec, int32_t* __restrict__ kcol) {
  givens_body(j, cs, h1, h2, ld, c0, ncols, rec, kcol);
}

// Back substitution R y = g for the k steps each column took.
__device__ __forceinline__ void backsolve_body(int ld, int c0, int ncols, double* __restrict__ rec,
                                               const int32_t* __restrict__ kcol) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c0 + ncols) return;
  double* R = rec + (size_t)c * kRec;
  const double* H = R;
  const double* g = R + kRecG;
  double* y = R + kRecY;
  const int k = kcol[c];
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int m = i + 1; m < k; ++m) s -= H[i * kMaxIter + m] * y[m];
    y[i] = s / H[i * kMaxIter + i];
  }
}

__global__ void k_backsolve(int ld, int c0, int ncols, double* __restrict__ rec, const int32_t* __restrict__ kcol) {
  backsolve_body(ld, c0, ncols, rec, kcol);
}

// X[r][lo + c] += sum_{i < k_c} y_i[c] Z_i[r][c] (grid-stride).
template <typename T>
__device__ __forceinline__ void update_x_body(const T* __restrict__ Z, size_t zstride, const double* __restrict__ rec,
                                              const int32_t* __restrict__ kcol, T* __restrict__ X, int ldx, int lo,
                                              int nrows, int ld, int c0, int ncols) {
  const long long total = (long long)nrows * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    const int k = kcol[c];
    if (k == 0) continue;
    const double* y = rec + (size_t)c * kRec + kRecY;
    T acc = 0;
    for (int i = 0; i < k; ++i) acc += (T)y[i] * Z[(size_t)i * zstride + (size_t)r * ld + c];
    X[(size_t)r * ldx + lo + c] += acc;
  }
}

template <typename T>
__global__ void k_update_x(const T* __restrict__ Z, size_t zstride, const double* __restrict__ rec,
                           const int32_t* __restrict__ kcol, T* __restrict__ X, int ldx, int lo, int nrows, int ld,
                           int c0, int ncols) {
  update_x_body<T>(Z, zstride, rec, kcol, X, ldx, lo, nrows, ld, c0, ncols);
}

// Mixed precision: X64[r][lo + c] += sum_{i < k_c} y_i[c] Z_i[r][c], the correction
// accumulated in FP32 and added to the FP64 state (iterative refinement per sweep).
__device__ __forceinline__ void update_x_mixed_body(const float* __restrict__ Z, size_t zstride,
                                                    const double* __restrict__ rec, const int32_t* __restrict__ kcol,
                                                    double* __restrict__ X, int ldx, int lo, int nrows, int ld,
                                                    int c0, int ncols) {
  const long long total = (long long)nrows * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    const int k = kcol[c];
    if (k == 0) continue;
    const double* y = rec + (size_t)c * kRec + kRecY;
    float acc = 0.f;
    for (int i = 0; i < k; ++i) acc += (float)y[i] * Z[(size_t)i * zstride + (size_t)r * ld + c];
    X[(size_t)r * ldx + lo + c] += (double)acc;
  }
}

__global__ void k_update_x_mixed(const float* __restrict__ Z, size_t zstride, const double* __restrict__ rec,
                                 const int32_t* __restrict__ kcol, double* __restrict__ X, int ldx, int lo, int nrows,
                                 int ld, int c0, int ncols) {
  update_x_mixed_body(Z, zstride, rec, kcol, X, ldx, lo, nrows, ld, c0, ncols);
}

// The same update with the columns' coefficients y converted to FP32 once per block (shared
// memory) instead of once per element, blocks owning row ranges and threads the columns
// (same per-element arithmetic: acc += y_i z_i in FP32, i ascending, then X += acc in FP64).
// Needs ncols <= kUpdCols.
constexpr int kUpdCols = 256;
__global__ void __launch_bounds__(256)
k_update_x_mixed_rows(const float* __restrict__ Z, size_t zstride, const double* __restrict__ rec,
                      const int32_t* __restrict__ kcol, double* __restrict__ X, int ldx, int lo, int nrows, int ld,
                      int c0, int ncols) {
  __shared__ float ys[kMaxIter][kUpdCols];
  __shared__ int ks[kUpdCols];
  for (int t = threadIdx.x; t < ncols; t += blockDim.x) {
    const int k = kcol[c0 + t];
    ks[t] = k;
    const double* y = rec + (size_t)(c0 + t) * kRec + kRecY;
    for (int i = 0; i < k; ++i) ys[i][t] = (float)y[i];
  }
  __syncthreads();
  const int per = (nrows + gridDim.x - 1) / gridDim.x;
  const int rb = blockIdx.x * per, re = min(nrows, rb + per);
  for (int r = rb; r < re; ++r) {
    for (int t = threadIdx.x; t < ncols; t += blockDim.x) {
      const int k = ks[t];
      if (k == 0) continue;
      const int c = c0 + t;
      float acc = 0.f;
      for (int i = 0; i < k; ++i) acc += ys[i][t] * Z[(size_t)i * zstride + (size_t)r * ld + c];
      X[(size_t)r * ldx + lo + c] += (double)acc;
    }
  }
}

// ---- batched variants: instance = blockIdx.z, arguments from the instance table ----

enum RedDst { RD_RES = 0, RD_WN0, RD_H1, RD_H2, RD_WW };

__global__ void kb_reduce(const InstDev* __restrict__ tab, int dst, int nslots) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active) return;
  const int ld = I.wcap;
  double* out = I.colscal;
  int c0 = I.c0, nc = I.nf;
  switch (dst) {
    case RD_RES: out = I.colscal + CS_RR * ld; c0 = 0; nc = I.nres; break;
    case RD_WN0: out = I.colscal + CS_WN0 * ld; break;
    case RD_H1: out = I.hvec; break;
    case RD_H2: out = I.hvec + (size_t)(kMaxIter + 1) * ld; break;
    default: out = I.colscal + CS_WW * ld; break;
  }
  if (nc <= 0) return;
  reduce_body(I.part, kRedBlocks, nslots, ld, c0, nc, out, ld);
}

__global__ void kb_fgmres_init(const InstDev* __restrict__ tab) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  fgmres_init_body(I.colscal, I.wcap, I.c0, I.nf, I.H, I.kcol);
}

// V_{j} = src * invh; src = V_0 (j = 0, in place) or w.
__global__ void kb_scale(const InstDev* __restrict__ tab, int j) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  const size_t vs = (size_t)I.n_dof * I.wcap;
  const float* src = j == 0 ? I.V : I.Wv;
  scale_cols_body<float>(src, I.V + j * vs, I.colscal + CS_INVH * I.wcap, I.n_dof, I.wcap, I.c0, I.nf);
}

// blockIdx.y = basis vector index; nvec = 0 computes |w|^2.
__global__ void __launch_bounds__(256) kb_dots(const InstDev* __restrict__ tab, int nvec) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  const size_t vs = (size_t)I.n_dof * I.wcap;
  if (nvec == 0) dots_body<float>(I.Wv, vs, I.Wv, I.n_dof, I.wcap, I.c0, I.nf, I.part);
  else dots_body<float>(I.V, vs, I.Wv, I.n_dof, I.wcap, I.c0, I.nf, I.part);
}

__global__ void kb_gs_axpy(const InstDev* __restrict__ tab, int nvec, int pass) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  const size_t vs = (size_t)I.n_dof * I.wcap;
  const double* h = I.hvec + (pass == 0 ? 0 : (size_t)(kMaxIter + 1) * I.wcap);
  gs_axpy_body<float>(I.V, vs, nvec, h, I.Wv, I.n_dof, I.wcap, I.c0, I.nf);
}

__global__ void kb_givens(const InstDev* __restrict__ tab, int j) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  givens_body(j, I.colscal, I.hvec, I.hvec + (size_t)(kMaxIter + 1) * I.wcap, I.wcap, I.c0, I.nf, I.H, I.kcol);
}

__global__ void kb_backsolve(const InstDev* __restrict__ tab) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  backsolve_body(I.wcap, I.c0, I.nf, I.H, I.kcol);
}

__global__ void kb_update_x(const InstDev* __restrict__ tab) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  update_x_mixed_body(I.Z, (size_t)I.n_dof * I.wcap, I.H, I.kcol, I.X64w, I.ldx, I.lo, I.n_dof, I.wcap, I.c0, I.nf);
}

}  // namespace

int krylov_record_doubles() { return kRec; }

void reduce_partials(biot_ctx* ctx, int nslots, int ncols, double* out, int ldo, int c0, int nblocks) {
  dim3 grid(div_up(ncols, 8), nslots);
  BIOT_LAUNCH(k_reduce_warp, grid, 256, 0, ctx->stream, ctx->part, nblocks, nslots, ctx->wcap, c0, ncols, out, ldo);
}

template <typename T> struct KBufs;
template <> struct KBufs<double> {
  static double* V(biot_ctx* c) { return c->V; }
  static double* Z(biot_ctx* c) { return c->Z; }
  static double* W(biot_ctx* c) { return c->Wv; }
};
template <> struct KBufs<float> {
  static float* V(biot_ctx* c) { return c->lp.V; }
  static float* Z(biot_ctx* c) { return c->lp.Z; }
  static float* W(biot_ctx* c) { return c->lp.Wv; }
};

template <typename T>
biot_status fgmres_cycle(biot_ctx* ctx, int lo, int c0, int ncols) {
  if (ncols <= 0) return BIOT_OK;
  cudaStream_t s = ctx->stream;
  const int ld = ctx->wcap, nd = ctx->n_dof;
  const size_t vs = (size_t)nd * ld;
  T* V = KBufs<T>::V(ctx);
  T* Z = KBufs<T>::Z(ctx);
  T* Wv = KBufs<T>::W(ctx);
  double* cs = ctx->colscal;
  double* h1 = ctx->hvec;
  double* h2 = ctx->hvec + (size_t)(kMaxIter + 1) * ld;
  const int cblk = div_up(ncols, 128);
  const int eblk = std::min(div_up((long long)nd * ncols, 256), 8192);
  // FP32: 16-byte vector kernels (memory-bound; rows of every [n_dof][ld] array must start on
  // 16-byte boundaries). FP64: the scalar kernels, which already run at the FP64 pipe's rate
  // (one FMA per loaded element) with more CTAs in flight; the vector forms measured slower.
  const bool vec = sizeof(T) == 4 && ld % KVec<T>::n == 0;
  const int vblk = std::min(div_up((long long)nd * div_up(ncols + KVec<T>::n, KVec<T>::n), 256), 8192);
  auto scale_cols = [&](const T* src, T* dst) {
    if (vec) BIOT_LAUNCH(k_scale_cols_vec<T>, vblk, 256, 0, s, src, dst, cs + CS_INVH * ld, nd, ld, c0, ncols);
    else BIOT_LAUNCH(k_scale_cols<T>, eblk, 256, 0, s, src, dst, cs + CS_INVH * ld, nd, ld, c0, ncols);
  };
  auto dots = [&](const T* Vb, int nvec, const T* w) {
    if (vec) BIOT_LAUNCH(k_dots_vec<T>, kDotBlocks, 256, 0, s, Vb, vs, nvec, w, nd, ld, c0, ncols, ctx->part);
    else BIOT_LAUNCH(k_dots<T>, dim3(kRedBlocks, nvec), 256, 0, s, Vb, vs, w, nd, ld, c0, ncols, ctx->part);
  };
  BIOT_LAUNCH(k_fgmres_init, cblk, 128, 0, s, cs, ld, c0, ncols, ctx->H, ctx->kcol);
  scale_cols(V, V);
  for (int j = 0; j < ctx->n_iter; ++j) {
    T* Vj = V + j * vs;
    T* Zj = Z + j * vs;
    precond_apply<T>(ctx, Vj, Zj, c0, ncols);
    launch_spmm_scaled<T>(ctx, Zj, Wv, c0, ncols);
    reduce_partials(ctx, 1, ncols, cs + CS_WN0 * ld, ld, c0, spmm_blocks(ctx));
    const bool fused = vec && j + 1 <= kFuseVecs;
    for (int pass = 0; pass < 2; ++pass) {
      double* h = pass == 0 ? h1 : h2;
      if (fused && pass == 1) {
        // the fused first update formed the partials
        reduce_partials(ctx, j + 1, ncols, h, ld, c0, j + 1 <= kDotChunk ? kDotBlocks : kRedBlocks);
        BIOT_LAUNCH((k_gs_axpy_rows_vec<T, true>), 2 * kRedBlocks, 256, 0, s, V, vs, j + 1, h, Wv, nd, ld, c0,
                    ncols, ctx->part);
        continue;
      }
      dots(V, j + 1, Wv);
      reduce_partials(ctx, j + 1, ncols, h, ld, c0, vec ? kDotBlocks : kRedBlocks);
      if (fused)  // pass 0: w -= V h1 and the partials of V^T w for h2 in one pass over V
        if (j + 1 <= kDotChunk)
          BIOT_LAUNCH(k_gs_axpy_dots_smem<T>, kDotBlocks, 256, 0, s, V, vs, j + 1, h, Wv, nd, ld, c0, ncols,
                      ctx->part);
        else
          BIOT_LAUNCH((k_gs_axpy_dots_vec<T, kFuseVecs>), kRedBlocks, 256, 0, s, V, vs, j + 1, h, Wv, nd, ld, c0,
                      ncols, ctx->part);
      else if (vec && pass == 0)
        BIOT_LAUNCH((k_gs_axpy_rows_vec<T, false>), 2 * kRedBlocks, 256, 0, s, V, vs, j + 1, h, Wv, nd, ld, c0,
                    ncols, ctx->part);
      else if (vec)  // the second sweep also forms the partial norms of the new w (2 x kRedBlocks
                     // partials: the first two slots of the partial-sum buffer)
        BIOT_LAUNCH((k_gs_axpy_rows_vec<T, true>), 2 * kRedBlocks, 256, 0, s, V, vs, j + 1, h, Wv, nd, ld, c0,
                    ncols, ctx->part);
      else BIOT_LAUNCH(k_gs_axpy<T>, eblk, 256, 0, s, V, vs, j + 1, h, Wv, nd, ld, c0, ncols);
    }
    if (!vec) dots(Wv, 1, Wv);
    reduce_partials(ctx, 1, ncols, cs + CS_WW * ld, ld, c0, vec ? 2 * kRedBlocks : kRedBlocks);
    BIOT_LAUNCH(k_givens, cblk, 128, 0, s, j, cs, h1, h2, ld, c0, ncols, ctx->H, ctx->kcol);
    if (j + 1 < ctx->n_iter) scale_cols(Wv, V + (j + 1) * vs);
  }
  BIOT_LAUNCH(k_backsolve, cblk, 128, 0, s, ld, c0, ncols, ctx->H, ctx->kcol);
  if (sizeof(T) == 8)
    BIOT_LAUNCH(k_update_x<double>, eblk, 256, 0, s, (const double*)Z, vs, ctx->H, ctx->kcol, ctx->X, ctx->ldx, lo, nd,
                ld, c0, ncols);
  else if (ncols <= kUpdCols)
    BIOT_LAUNCH(k_update_x_mixed_rows, 4 * 152, 256, 0, s, (const float*)Z, vs, ctx->H, ctx->kcol, ctx->X, ctx->ldx,
                lo, nd, ld, c0, ncols);
  else
    BIOT_LAUNCH(k_update_x_mixed, eblk, 256, 0, s, (const float*)Z, vs, ctx->H, ctx->kcol, ctx->X, ctx->ldx, lo, nd,
                ld, c0, ncols);
  BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

template biot_status fgmres_cycle<double>(biot_ctx*, int, int, int);

// One FGMRES(n_iter) cycle for every instance of a batch (windows in the table).
// The launch sequence depends only on n_iter, so it can be captured in a CUDA graph.
void batched_fgmres_cycle(const InstDev* tab, int count, int n_iter, int max_wcap, int max_ndof, int max_band,
                          bool bf16, bool tri, cudaStream_t s, GmgBatch* gb) {
  const int cblk = div_up(max_wcap, 128);
  const int eblk = std::min(div_up((long long)max_ndof * max_wcap, 256), 2048);
  BIOT_LAUNCH(kb_fgmres_init, dim3(cblk, 1, count), 128, 0, s, tab);
  BIOT_LAUNCH(kb_scale, dim3(eblk, 1, count), 256, 0, s, tab, 0);
  for (int j = 0; j < n_iter; ++j) {
    if (gb) gmg_batch_apply(gb, tab, count, j, tri, s);
    else batched_precond_apply(tab, count, j, max_wcap, max_band, tri, s);
    launch_batched_spmm(tab, count, bf16, j, s);
    BIOT_LAUNCH(kb_reduce, dim3(cblk, 1, count), 128, 0, s, tab, (int)RD_WN0, 1);
    for (int pass = 0; pass < 2; ++pass) {
      BIOT_LAUNCH(kb_dots, dim3(kRedBlocks, j + 1, count), 256, 0, s, tab, j + 1);
      BIOT_LAUNCH(kb_reduce, dim3(cblk, j + 1, count), 128, 0, s, tab, (int)(pass == 0 ? RD_H1 : RD_H2), j + 1);
      BIOT_LAUNCH(kb_gs_axpy, dim3(eblk, 1, count), 256, 0, s, tab, j + 1, pass);
    }
    BIOT_LAUNCH(kb_dots, dim3(kRedBlocks, 1, count), 256, 0, s, tab, 0);
    BIOT_LAUNCH(kb_reduce, dim3(cblk, 1, count), 128, 0, s, tab, (int)RD_WW, 1);
    BIOT_LAUNCH(kb_givens, dim3(cblk, 1, count), 128, 0, s, tab, j);
    if (j + 1 < n_iter) BIOT_LAUNCH(kb_scale, dim3(eblk, 1, count), 256, 0, s, tab, j + 1);
  }
  BIOT_LAUNCH(kb_backsolve, dim3(cblk, 1, count), 128, 0, s, tab);
  BIOT_LAUNCH(kb_update_x, dim3(eblk, 1, count), 256, 0, s, tab);
}

void batched_residual_reduce(const InstDev* tab, int count, int max_wcap, cudaStream_t s) {
  BIOT_LAUNCH(kb_reduce, dim3(div_up(max_wcap, 128), 2, count), 128, 0, s, tab, (int)RD_RES, 2);
}


template biot_status fgmres_cycle<float>(biot_ctx*, int, int, int);

}  // namespace biot
