// Geometric multigrid V-cycles for the preconditioner's blocks A and S (biot_set_inner_solver).
//
// Sec. 3.1 builds P1 and P2 from solves with A and S = tau C + beta L and leaves open how they
// are done; Sec. 4's meshes come from joining edge midpoints, so the uniform meshes of sizes
// n, n/2, n/4, ... are nested and their P1 spaces too. This file runs the inexact alternative
// to the exact (band / substructured) block solves: V-cycles on that hierarchy, as streaming
// multi-right-hand-side kernels over every active time step at once.
//
// * Level 0 is the context's own mesh. Level l >= 1 is a context of its own on the n / 2^l
//   mesh, assembled from the same problem with the element permeability averaged over the
//   four fine children of each coarse triangle and the fine level's beta: for P1 on nested
//   meshes that is the Galerkin operator P^T K P exactly (coarse basis gradients are constant
//   on a coarse triangle; A's coefficients and beta L are constant).
// * Every level's block-diagonal operator diag(A, S) is kept as a 7-point stencil per node
//   (the "/"-split mesh couples (i, j) with (i +- 1, j), (i, j +- 1), (i - 1, j - 1),
//   (i + 1, j + 1)): 2 x 2 blocks of A, scalars of S, and the inverses of the node's diagonal
//   blocks (the smoother's preconditioner M).
// * Smoother: Chebyshev on M^{-1} K over [lam / 8, 1.1 lam], lam from 20 power steps on
//   M^{-1} K from the checkerboard vector; Dirichlet rows (identity rows, decoupled) are solved
//   exactly (x = b). Restriction P^T (coarse Dirichlet rows zeroed), prolongation by linear
//   interpolation; the coarsest level is solved exactly by its band factors.
// * Vectors keep the node-interleaved layout [3 nn][ldg] (time step fastest, ldg = window
//   capacity rounded up to four columns); a V-cycle on A touches rows 3v, 3v+1, on S rows
//   3v+2, and P2 runs both in one pass. A thread owns one node and 16 bytes of columns.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace biot {

namespace {

// Per node (160 bytes in FP32, read as ten 16-byte vectors): A's 7 blocks 2 x 2 at 0..27,
// M_u^{-1} (2 x 2) at 28..31, S's 7 entries at 32..38, M_p^{-1} at 39.
constexpr int kCoef = 40;
constexpr int kCoefMu = 28, kCoefP = 32, kCoefMp = 39;
constexpr int kMinCoarse = 16;    // coarsen while n is even and above this
constexpr double kChebLowDiv = 8.0;
constexpr int kPowerIters = 20;
constexpr int kThreads = 256;
constexpr int kMaxSmooth = 8;

enum GmgBuf { GB_B = 0, GB_X, GB_XA, GB_XB, GB_D, GB_R, GB_E, kGmgBufs };

template <typename T> struct V16;
template <> struct V16<float> {
  using V = float4;
  static constexpr int n = 4;
  __device__ static void get(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ static V make(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <> struct V16<double> {
  using V = double2;
  static constexpr int n = 2;
  __device__ static void get(const V& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ static V make(const double* o) { return make_double2(o[0], o[1]); }
};

template <typename T> __device__ __forceinline__ void ldv(const T* p, T* o) {
  V16<T>::get(*reinterpret_cast<const typename V16<T>::V*>(p), o);
}
template <typename T> __device__ __forceinline__ void stv(T* p, const T* o) {
  *reinterpret_cast<typename V16<T>::V*>(p) = V16<T>::make(o);
}

// Neighbour k of node (i, j) on the "/"-split mesh, k = 0..6 in ascending node order:
// (i-1, j-1), (i, j-1), (i-1, j), (i, j), (i+1, j), (i, j+1), (i+1, j+1); -1 if absent.
__host__ __device__ __forceinline__ int nbr_of(int k, int i, int j, int n) {
  const int nx = n + 1;
  switch (k) {
    case 0: return (i > 0 && j > 0) ? (j - 1) * nx + i - 1 : -1;
    case 1: return j > 0 ? (j - 1) * nx + i : -1;
    case 2: return i > 0 ? j * nx + i - 1 : -1;
    case 3: return j * nx + i;
    case 4: return i < n ? j * nx + i + 1 : -1;
    case 5: return j < n ? (j + 1) * nx + i : -1;
    default: return (i < n && j < n) ? (j + 1) * nx + i + 1 : -1;
  }
}

// Stencil of diag(A, S) from the eliminated CSR of AA (rows of node v: three runs of deg(v)
// triples): A's 2 x 2 blocks, S = -AA_pp, and the inverted node-diagonal blocks.
__global__ void k_gmg_stencil(int n, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
                              const int32_t* __restrict__ rowptr, const double* __restrict__ val,
                              double* __restrict__ coef) {
  const int nx = n + 1, nn = nx * nx;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
    double* cf = coef + (size_t)v * kCoef;
    for (int q = 0; q < kCoef; ++q) cf[q] = 0.0;
    const int32_t np = nodeptr[v];
    const int deg = nodeptr[v + 1] - np;
    const int32_t r0 = rowptr[3 * v], r1 = r0 + 3 * deg, r2 = r1 + 3 * deg;
    for (int k = 0; k < deg; ++k) {
      const int m = nbr[np + k];
      const int d = m - v;
      int slot = -1;
      if (d == -(n + 2)) slot = 0;
      else if (d == -(n + 1)) slot = 1;
      else if (d == -1) slot = 2;
      else if (d == 0) slot = 3;
      else if (d == 1) slot = 4;
      else if (d == n + 1) slot = 5;
      else if (d == n + 2) slot = 6;
      if (slot < 0) continue;  // no other couplings exist on this mesh
      cf[slot * 4 + 0] = val[r0 + 3 * k];
      cf[slot * 4 + 1] = val[r0 + 3 * k + 1];
      cf[slot * 4 + 2] = val[r1 + 3 * k];
      cf[slot * 4 + 3] = val[r1 + 3 * k + 1];
      cf[kCoefP + slot] = -val[r2 + 3 * k + 2];
    }
    const double a = cf[12], b = cf[13], c = cf[14], e = cf[15];
    const double det = a * e - b * c;
    cf[kCoefMu + 0] = e / det;
    cf[kCoefMu + 1] = -b / det;
    cf[kCoefMu + 2] = -c / det;
    cf[kCoefMu + 3] = a / det;
    cf[kCoefMp] = 1.0 / cf[kCoefP + 3];
  }
}

__global__ void k_gmg_to_f32(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Coarse element permeability: the mean of the four fine children (triangle 2 (j n + i) is the
// lower, 2 (j n + i) + 1 the upper triangle of cell (i, j)).
__global__ void k_gmg_coarsen_kappa(int nf, const double* __restrict__ kf, double* __restrict__ kc) {
  const int nc = nf / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * nc * nc; e += gridDim.x * blockDim.x) {
    const int cell = e >> 1, I = cell % nc, J = cell / nc;
    const int i = 2 * I, j = 2 * J;
    auto lo = [&](int ii, int jj) { return kf[2 * (jj * nf + ii)]; };
    auto up = [&](int ii, int jj) { return kf[2 * (jj * nf + ii) + 1]; };
    kc[e] = (e & 1) ? (up(i, j) + up(i, j + 1) + up(i + 1, j + 1) + lo(i, j + 1)) / 4.0
                    : (lo(i, j) + lo(i + 1, j) + lo(i + 1, j + 1) + up(i + 1, j)) / 4.0;
  }
}

// ---- setup: power method on M^{-1} K for one block (FP64, one vector) ----

// x = (-1)^(i + j) on every field of block `blk` (0: A, 2 DOFs per node; 1: S).
__global__ void k_gmg_checker(int n, int blk, double* __restrict__ x) {
  const int nx = n + 1, d = blk == 0 ? 2 : 1, N = nx * nx * d;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) {
    const int v = q / d, i = v % nx, j = v / nx;
    x[q] = ((i + j) & 1) ? -1.0 : 1.0;
  }
}

__global__ void k_gmg_div(double* __restrict__ x, int N, const double* __restrict__ nrm) {
  const double s = *nrm;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) x[q] = x[q] / s;
}

// y = M^{-1} K x for block blk (vectors in block order: 2 v + f for A, v for S).
__global__ void k_gmg_power_apply(int n, int blk, const double* __restrict__ coef, const double* __restrict__ x,
                                  double* __restrict__ y) {
  const int nx = n + 1, nn = nx * nx;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
    const double* cf = coef + (size_t)v * kCoef;
    const int j = v / nx, i = v - j * nx;
    if (blk == 0) {
      double y0 = 0.0, y1 = 0.0;
      for (int k = 0; k < 7; ++k) {
        const int m = nbr_of(k, i, j, n);
        if (m < 0) continue;
        y0 += cf[4 * k] * x[2 * m] + cf[4 * k + 1] * x[2 * m + 1];
        y1 += cf[4 * k + 2] * x[2 * m] + cf[4 * k + 3] * x[2 * m + 1];
      }
      y[2 * v] = cf[kCoefMu] * y0 + cf[kCoefMu + 1] * y1;
      y[2 * v + 1] = cf[kCoefMu + 2] * y0 + cf[kCoefMu + 3] * y1;
    } else {
      double s = 0.0;
      for (int k = 0; k < 7; ++k) {
        const int m = nbr_of(k, i, j, n);
        if (m >= 0) s += cf[kCoefP + k] * x[m];
      }
      y[v] = cf[kCoefMp] * s;
    }
  }
}

// |x|^2: per-block partial sums (fixed grid), then one block sums them in order and takes
// the square root.
__global__ void k_gmg_norm_part(const double* __restrict__ x, int N, double* __restrict__ part) {
  __shared__ double sm[kThreads];
  double s = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) s += x[q] * x[q];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void k_gmg_norm_fin(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *out = sqrt(s);
  }
}

// ---- the V-cycle's kernels: FM = fields (1: A's rows 3v, 3v+1; 2: S's rows 3v+2; 3: both) ----

// Level-0 right-hand side from the Krylov vector (scaled by |diag AA|^{1/2}); mode 0: A rows
// b = vin dsq; 1: S rows b = -vin dsq (P2's z_p = -S^{-1} r_p); 2: S rows b = tp (P1); 3: 0 and 1.
// A thread owns one node and 16 bytes of columns of b (all ldg columns: those outside
// [c0, c0 + ncols) are set to zero, which keeps the level buffers finite).
template <typename T>
__device__ __forceinline__ void prep_body(int nn, int mode, const T* __restrict__ vin, const double* __restrict__ dsq,
                                          const T* __restrict__ tp, T* __restrict__ b, int ld, int ldg, int c0,
                                          int ncols) {
  constexpr int VEC = V16<T>::n;
  const int nch = ldg / VEC;
  const int total = nn * nch;
  const bool vec_in = ld % VEC == 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int v = q / nch, c = (q - v * nch) * VEC;
    const bool full = vec_in && c >= c0 && c + VEC <= c0 + ncols;
    auto load = [&](const T* row, T* o) {
      if (full) {
        ldv(row + c, o);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) o[k] = (c + k >= c0 && c + k < c0 + ncols) ? row[c + k] : T(0);
      }
    };
    T a[VEC];
    if (mode == 0 || mode == 3) {
      for (int f = 0; f < 2; ++f) {
        load(vin + (size_t)(3 * v + f) * ld, a);
        const T sc = (T)dsq[3 * v + f];  // one conversion per row: FP64 work per element is slow here
#pragma unroll
        for (int k = 0; k < VEC; ++k) a[k] *= sc;
        stv(b + (size_t)(3 * v + f) * ldg + c, a);
      }
    }
    if (mode == 1 || mode == 3) {
      load(vin + (size_t)(3 * v + 2) * ld, a);
      const T sc = -(T)dsq[3 * v + 2];
#pragma unroll
      for (int k = 0; k < VEC; ++k) a[k] *= sc;
      stv(b + (size_t)(3 * v + 2) * ldg + c, a);
    }
    if (mode == 2) {
      load(tp + (size_t)v * ld, a);
      stv(b + (size_t)(3 * v + 2) * ldg + c, a);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gmg_prep(int nn, int mode, const T* __restrict__ vin, const double* __restrict__ dsq, const T* __restrict__ tp,
           T* __restrict__ b, int ld, int ldg, int c0, int ncols) {
  prep_body<T>(nn, mode, vin, dsq, tp, b, ld, ldg, c0, ncols);
}

// z rows of the fields in FM from the V-cycle's level-0 result.
template <typename T, int FM>
__global__ void k_gmg_finish(int nn, const T* __restrict__ x, T* __restrict__ z, int ld, int ldg, int c0, int ncols) {
  const long long total = (long long)nn * ncols;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(q / ncols), c = c0 + (int)(q % ncols);
    if (FM & 1) {
      z[(size_t)(3 * v) * ld + c] = x[(size_t)(3 * v) * ldg + c];
      z[(size_t)(3 * v + 1) * ld + c] = x[(size_t)(3 * v + 1) * ldg + c];
    }
    if (FM & 2) z[(size_t)(3 * v + 2) * ld + c] = x[(size_t)(3 * v + 2) * ldg + c];
  }
}

// Columns c .. c + VEC - 1 of one row of z (row start `row`): a 16-byte store when the chunk lies
// inside [c0, c0 + ncols) and ldo keeps rows 16-byte aligned, else element by element.
template <typename T>
__device__ __forceinline__ void store_out(T* row, const T* x, int c, int ldo, int c0, int ncols) {
  constexpr int VEC = V16<T>::n;
  if (ldo % VEC == 0 && c >= c0 && c + VEC <= c0 + ncols) {
    stv(row + c, x);
  } else {
#pragma unroll
    for (int q = 0; q < VEC; ++q)
      if (c + q >= c0 && c + q < c0 + ncols) row[c + q] = x[q];
  }
}

// Four consecutive coefficients (16-byte aligned) as one or two vector loads.
template <typename T> __device__ __forceinline__ void ld4(const T* p, T* o) {
  if (sizeof(T) == 4) {
    ldv(p, o);
  } else {
    ldv(p, o);
    ldv(p + 2, o + 2);
  }
}

// K x for the rows in FM of node v (i, j), columns c .. c + VEC - 1.
template <typename T, int FM>
__device__ __forceinline__ void stencil_apply(const T* __restrict__ cf, const T* __restrict__ x, int i, int j, int n,
                                              int ldg, int c, T* y0, T* y1, T* y2) {
  constexpr int VEC = V16<T>::n;
#pragma unroll
  for (int q = 0; q < VEC; ++q) y0[q] = y1[q] = y2[q] = T(0);
  T sp[8];
  if (FM & 2) {
    ld4(cf + kCoefP, sp);
    ld4(cf + kCoefP + 4, sp + 4);
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int m = nbr_of(k, i, j, n);
    if (m < 0) continue;
    const T* xm = x + (size_t)(3 * m) * ldg + c;
    if (FM & 1) {
      T a[VEC], b[VEC], cc[4];
      ldv(xm, a);
      ldv(xm + ldg, b);
      ld4(cf + 4 * k, cc);
      const T c00 = cc[0], c01 = cc[1], c10 = cc[2], c11 = cc[3];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        y0[q] += c00 * a[q] + c01 * b[q];
        y1[q] += c10 * a[q] + c11 * b[q];
      }
    }
    if (FM & 2) {
      T p[VEC];
      ldv(xm + 2 * ldg, p);
      const T cp = sp[k];
#pragma unroll
      for (int q = 0; q < VEC; ++q) y2[q] += cp * p[q];
    }
  }
}

// One Chebyshev step on the rows in FM: s = M^{-1} (b - K x_in) (x_in = 0: ZERO), d = c1 d + c2 s
// (READD false: c1 d dropped), x_out = x_in + d; Dirichlet rows x_out = b, d = 0.
// OUTZ: x_out is the preconditioner's output z (leading dimension ldo, only the columns
// [c0, c0 + ncols) written, 16-byte stores when ldo allows) instead of a level buffer.
// DMODE bit 0 (DM_FROM_X): the previous increment is read from x_in, which holds it after a
// step from zero (x = 0 + d; on Dirichlet rows x = b but d is not used there); bit 1
// (DM_NO_STORE): the new increment is not stored (no later step of the cycle reads it).
// Each saves one pass over a level vector.
enum { DM_FROM_X = 1, DM_NO_STORE = 2 };
template <typename T, int FM, bool ZERO, bool READD, bool OUTZ, int DMODE = 0>
__device__ __forceinline__ void smooth_body(int n, const T* __restrict__ coef, const uint8_t* __restrict__ dmask,
                                            const T* __restrict__ xin, const T* __restrict__ b, T* __restrict__ d,
                                            T* __restrict__ xout, T cu1, T cu2, T cp1, T cp2, int ldg, int ca,
                                            int nch, int ldo, int c0, int ncols) {
  constexpr int VEC = V16<T>::n;
  const int nx = n + 1;
  // 32-bit work index: the set-up keeps nodes x column chunks below 2^31
  const int total = nx * nx * nch;
  // grid-stride over (node, column chunk) in the natural node order: the whole grid works on a
  // band of a few mesh rows at a time, so the neighbour rows a step needs were read one or two
  // steps before and are still in L2 (contiguous ranges per CTA kept the whole level live and
  // read x from DRAM about three times)
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int v = q / nch, c = ca + (q - v * nch) * VEC;
    const int j = v / nx, i = v - j * nx;
    const T* cf = coef + (size_t)v * kCoef;
    T y0[VEC], y1[VEC], y2[VEC];
    if (!ZERO) {
      stencil_apply<T, FM>(cf, xin, i, j, n, ldg, c, y0, y1, y2);
    } else {
#pragma unroll
      for (int k = 0; k < VEC; ++k) y0[k] = y1[k] = y2[k] = T(0);
    }
    const size_t r0 = (size_t)(3 * v) * ldg + c;
    if (FM & 1) {
      T b0[VEC], b1[VEC], x0[VEC], x1[VEC], d0[VEC], d1[VEC];
      ldv(b + r0, b0);
      ldv(b + r0 + ldg, b1);
      if (!ZERO) {
        ldv(xin + r0, x0);
        ldv(xin + r0 + ldg, x1);
      }
      if (READD && (DMODE & DM_FROM_X)) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          d0[k] = x0[k];
          d1[k] = x1[k];
        }
      } else if (READD) {
        ldv(d + r0, d0);
        ldv(d + r0 + ldg, d1);
      }
      T mu[4];
      ld4(cf + kCoefMu, mu);
      const T m00 = mu[0], m01 = mu[1], m10 = mu[2], m11 = mu[3];
      const bool dir0 = dmask[3 * v] != 0, dir1 = dmask[3 * v + 1] != 0;
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        const T r0v = b0[k] - y0[k], r1v = b1[k] - y1[k];
        const T s0 = m00 * r0v + m01 * r1v, s1 = m10 * r0v + m11 * r1v;
        T e0 = cu2 * s0, e1 = cu2 * s1;
        if (READD) {
          e0 = cu1 * d0[k] + e0;
          e1 = cu1 * d1[k] + e1;
        }
        const T xa = ZERO ? T(0) : x0[k], xb = ZERO ? T(0) : x1[k];
        x0[k] = dir0 ? b0[k] : xa + e0;
        x1[k] = dir1 ? b1[k] : xb + e1;
        d0[k] = dir0 ? T(0) : e0;
        d1[k] = dir1 ? T(0) : e1;
      }
      if (OUTZ) {
        store_out(xout + (size_t)(3 * v) * ldo, x0, c, ldo, c0, ncols);
        store_out(xout + (size_t)(3 * v + 1) * ldo, x1, c, ldo, c0, ncols);
      } else {
        stv(xout + r0, x0);
        stv(xout + r0 + ldg, x1);
      }
      if (!(DMODE & DM_NO_STORE)) {
        stv(d + r0, d0);
        stv(d + r0 + ldg, d1);
      }
    }
    if (FM & 2) {
      const size_t r2 = r0 + 2 * (size_t)ldg;
      T b2[VEC], x2[VEC], d2[VEC];
      ldv(b + r2, b2);
      if (!ZERO) ldv(xin + r2, x2);
      if (READD && (DMODE & DM_FROM_X)) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) d2[k] = x2[k];
      } else if (READD) {
        ldv(d + r2, d2);
      }
      const T mp = cf[kCoefMp];
      const bool dir2 = dmask[3 * v + 2] != 0;
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        T e = cp2 * (mp * (b2[k] - y2[k]));
        if (READD) e = cp1 * d2[k] + e;
        const T xa = ZERO ? T(0) : x2[k];
        x2[k] = dir2 ? b2[k] : xa + e;
        d2[k] = dir2 ? T(0) : e;
      }
      if (OUTZ) store_out(xout + (size_t)(3 * v + 2) * ldo, x2, c, ldo, c0, ncols);
      else stv(xout + r2, x2);
      if (!(DMODE & DM_NO_STORE)) stv(d + r2, d2);
    }
  }
}

template <typename T, int FM, bool ZERO, bool READD, bool OUTZ = false, int DMODE = 0>
__global__ void __launch_bounds__(kThreads)
k_gmg_smooth(int n, const T* __restrict__ coef, const uint8_t* __restrict__ dmask, const T* __restrict__ xin,
             const T* __restrict__ b, T* __restrict__ d, T* __restrict__ xout, T cu1, T cu2, T cp1, T cp2, int ldg,
             int ca, int nch, int ldo = 0, int c0 = 0, int ncols = 0) {
  smooth_body<T, FM, ZERO, READD, OUTZ, DMODE>(n, coef, dmask, xin, b, d, xout, cu1, cu2, cp1, cp2, ldg, ca, nch, ldo,
                                               c0, ncols);
}

// r = b - K x on the rows in FM.
template <typename T, int FM>
__device__ __forceinline__ void residual_body(int n, const T* __restrict__ coef, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ r, int ldg, int ca, int nch) {
  constexpr int VEC = V16<T>::n;
  const int nx = n + 1;
  // 32-bit work index: the set-up keeps nodes x column chunks below 2^31
  const int total = nx * nx * nch;
  // grid-stride over (node, column chunk) in the natural node order: the whole grid works on a
  // band of a few mesh rows at a time, so the neighbour rows a step needs were read one or two
  // steps before and are still in L2 (contiguous ranges per CTA kept the whole level live and
  // read x from DRAM about three times)
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int v = q / nch, c = ca + (q - v * nch) * VEC;
    const int j = v / nx, i = v - j * nx;
    T y0[VEC], y1[VEC], y2[VEC];
    stencil_apply<T, FM>(coef + (size_t)v * kCoef, x, i, j, n, ldg, c, y0, y1, y2);
    const size_t r0 = (size_t)(3 * v) * ldg + c;
    if (FM & 1) {
      T b0[VEC], b1[VEC];
      ldv(b + r0, b0);
      ldv(b + r0 + ldg, b1);
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        b0[k] -= y0[k];
        b1[k] -= y1[k];
      }
      stv(r + r0, b0);
      stv(r + r0 + ldg, b1);
    }
    if (FM & 2) {
      T b2[VEC];
      ldv(b + r0 + 2 * (size_t)ldg, b2);
#pragma unroll
      for (int k = 0; k < VEC; ++k) b2[k] -= y2[k];
      stv(r + r0 + 2 * (size_t)ldg, b2);
    }
  }
}

template <typename T, int FM>
__global__ void __launch_bounds__(kThreads)
k_gmg_residual(int n, const T* __restrict__ coef, const T* __restrict__ x, const T* __restrict__ b,
               T* __restrict__ r, int ldg, int ca, int nch) {
  residual_body<T, FM>(n, coef, x, b, r, ldg, ca, nch);
}

// Coarse right-hand side bc = P^T r on the rows in FM (coarse Dirichlet rows zero): fine node
// (2I, 2J) with weight 1, its six mesh neighbours (the midpoints of the coarse edges at (I, J))
// with weight 1/2.
template <typename T, int FM>
__device__ __forceinline__ void restrict_body(int nc, const T* __restrict__ r, const uint8_t* __restrict__ dmask_c,
                                              T* __restrict__ bc, int ldg, int ca, int nch) {
  constexpr int VEC = V16<T>::n;
  const int cx = nc + 1, nf = 2 * nc;
  // 32-bit work index: the set-up keeps nodes x column chunks below 2^31
  const int total = cx * cx * nch;
  // grid-stride in the natural order of the coarse nodes (the fine rows stay in L2)
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int V = q / nch, c = ca + (q - V * nch) * VEC;
    const int J = V / cx, i = 2 * (V - J * cx), j = 2 * J;
    T s0[VEC], s1[VEC], s2[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) s0[k] = s1[k] = s2[k] = T(0);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const int m = nbr_of(k, i, j, nf);
      if (m < 0) continue;
      const T w = k == 3 ? T(1) : T(0.5);
      const T* rm = r + (size_t)(3 * m) * ldg + c;
      T a[VEC];
      if (FM & 1) {
        ldv(rm, a);
#pragma unroll
        for (int e = 0; e < VEC; ++e) s0[e] += w * a[e];
        ldv(rm + ldg, a);
#pragma unroll
        for (int e = 0; e < VEC; ++e) s1[e] += w * a[e];
      }
      if (FM & 2) {
        ldv(rm + 2 * ldg, a);
#pragma unroll
        for (int e = 0; e < VEC; ++e) s2[e] += w * a[e];
      }
    }
    const size_t o = (size_t)(3 * V) * ldg + c;
    if (FM & 1) {
      if (dmask_c[3 * V]) for (int e = 0; e < VEC; ++e) s0[e] = T(0);
      if (dmask_c[3 * V + 1]) for (int e = 0; e < VEC; ++e) s1[e] = T(0);
      stv(bc + o, s0);
      stv(bc + o + ldg, s1);
    }
    if (FM & 2) {
      if (dmask_c[3 * V + 2]) for (int e = 0; e < VEC; ++e) s2[e] = T(0);
      stv(bc + o + 2 * (size_t)ldg, s2);
    }
  }
}

template <typename T, int FM>
__global__ void __launch_bounds__(kThreads)
k_gmg_restrict(int nc, const T* __restrict__ r, const uint8_t* __restrict__ dmask_c, T* __restrict__ bc, int ldg,
               int ca, int nch) {
  restrict_body<T, FM>(nc, r, dmask_c, bc, ldg, ca, nch);
}

// x += P xc on the rows in FM: linear interpolation of the coarse nodal values.
template <typename T, int FM>
__device__ __forceinline__ void prolong_body(int nf, const T* __restrict__ xc, T* __restrict__ x, int ldg, int ca,
                                             int nch) {
  constexpr int VEC = V16<T>::n;
  const int fx = nf + 1, cx = nf / 2 + 1;
  // 32-bit work index: the set-up keeps nodes x column chunks below 2^31
  const int total = fx * fx * nch;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int v = q / nch, c = ca + (q - v * nch) * VEC;
    const int j = v / fx, i = v - j * fx;
    int s0, s1;  // coarse source nodes (equal: one source)
    if (!(i & 1) && !(j & 1)) s0 = s1 = (j / 2) * cx + i / 2;
    else if (!(j & 1)) { s0 = (j / 2) * cx + (i - 1) / 2; s1 = s0 + 1; }
    else if (!(i & 1)) { s0 = ((j - 1) / 2) * cx + i / 2; s1 = s0 + cx; }
    else { s0 = ((j - 1) / 2) * cx + (i - 1) / 2; s1 = s0 + cx + 1; }
    const T w = s0 == s1 ? T(1) : T(0.5);
    for (int f = 0; f < 3; ++f) {
      if (f < 2 && !(FM & 1)) continue;
      if (f == 2 && !(FM & 2)) continue;
      T a[VEC], bq[VEC], xv[VEC];
      ldv(xc + (size_t)(3 * s0 + f) * ldg + c, a);
      ldv(xc + (size_t)(3 * s1 + f) * ldg + c, bq);
      T* xr = x + (size_t)(3 * v + f) * ldg + c;
      ldv(xr, xv);
#pragma unroll
      for (int e = 0; e < VEC; ++e) xv[e] += s0 == s1 ? a[e] : w * (a[e] + bq[e]);
      stv(xr, xv);
    }
  }
}

template <typename T, int FM>
__global__ void __launch_bounds__(kThreads)
k_gmg_prolong(int nf, const T* __restrict__ xc, T* __restrict__ x, int ldg, int ca, int nch) {
  prolong_body<T, FM>(nf, xc, x, ldg, ca, nch);
}

// x += e on the rows in FM (repeated V-cycles).
template <typename T, int FM>
__global__ void k_gmg_axpy(int nn, const T* __restrict__ e, T* __restrict__ x, int ldg, int ca, int nch) {
  constexpr int VEC = V16<T>::n;
  // 32-bit work index: the set-up keeps nodes x column chunks below 2^31
  const int total = nn * nch;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int v = q / nch, c = ca + (q - v * nch) * VEC;
    for (int f = 0; f < 3; ++f) {
      if ((f < 2 && !(FM & 1)) || (f == 2 && !(FM & 2))) continue;
      T a[VEC], xv[VEC];
      const size_t o = (size_t)(3 * v + f) * ldg + c;
      ldv(e + o, a);
      ldv(x + o, xv);
#pragma unroll
      for (int k = 0; k < VEC; ++k) xv[k] += a[k];
      stv(x + o, xv);
    }
  }
}

// The coarsest level's input to its exact P2 apply: vin = +-b d (so that P2^{-1} (vin / d)
// gives A^{-1} b_u and S^{-1} b_p); rows outside FM zero.
template <typename T, int FM>
__device__ __forceinline__ void coarse_prep_body(int nn, const T* __restrict__ b, const double* __restrict__ dsc,
                                                 T* __restrict__ vin, int ldg, int c0, int ncols) {
  const long long total = (long long)nn * ncols;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(q / ncols), c = c0 + (int)(q % ncols);
    for (int f = 0; f < 3; ++f) {
      const size_t o = (size_t)(3 * v + f) * ldg + c;
      const bool on = f < 2 ? (FM & 1) : (FM & 2);
      const T s = (T)(f < 2 ? dsc[3 * v + f] : -dsc[3 * v + f]);
      vin[o] = on ? b[o] * s : T(0);
    }
  }
}

template <typename T, int FM>
__global__ void k_gmg_coarse_prep(int nn, const T* __restrict__ b, const double* __restrict__ dsc,
                                  T* __restrict__ vin, int ldg, int c0, int ncols) {
  coarse_prep_body<T, FM>(nn, b, dsc, vin, ldg, c0, ncols);
}

int grid_for(long long work) {
  return (int)std::max<long long>(1, std::min<long long>((work + kThreads - 1) / kThreads, 152 * 16));
}
// The stencil kernels' grid: they walk their work grid-stride, so the grid must be resident at
// once to sweep the mesh as one band: four CTAs of 256 threads per SM (their 48-61 registers
// allow four; with eight the second wave re-read the first wave's band boundaries).
int grid_stencil(long long work) { return std::min(grid_for(work), 152 * 4); }

struct GmgLevel {
  int n = 0, nn = 0;
  biot_ctx* lc = nullptr;           // the level's own context (level 0: none, the fine context)
  double* coef64 = nullptr;         // [nn][kCoef]
  float* coef32 = nullptr;
  const uint8_t* dmask = nullptr;   // [3 nn]
  double lam[2] = {0.0, 0.0};       // power-method estimates of lam_max(M^{-1} K): A, S
  double c1[2][kMaxSmooth] = {};    // Chebyshev coefficients per block and step
  double c2[2][kMaxSmooth] = {};
  void* buf[kGmgBufs] = {};         // [3 nn][ldg] in the sweep precision
};

}  // namespace

struct Gmg {
  int L = 0, cycles = 1, smooth = 2, ldg = 0;
  bool fp64 = true;
  std::vector<GmgLevel> lv;
};

namespace {

biot_ctx* owner(biot_ctx* ctx, GmgLevel& L) { return L.lc ? L.lc : ctx; }

template <typename T> const T* coef_of(const GmgLevel& L);
template <> const double* coef_of<double>(const GmgLevel& L) { return L.coef64; }
template <> const float* coef_of<float>(const GmgLevel& L) { return L.coef32; }

template <typename T> T* buf_of(GmgLevel& L, int k) { return static_cast<T*>(L.buf[k]); }

biot_status norm_dev(biot_ctx* ctx, const double* x, int N, double* part, double* out_dev, double* out_host) {
  BIOT_LAUNCH(k_gmg_norm_part, kRedBlocks, kThreads, 0, ctx->stream, x, N, part);
  BIOT_LAUNCH(k_gmg_norm_fin, 1, 32, 0, ctx->stream, part, kRedBlocks, out_dev);
  if (out_host) {
    BIOT_CU(ctx, cudaMemcpyAsync(out_host, out_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return BIOT_OK;
}

// lam_max(M^{-1} K) of both blocks of one level: kPowerIters power steps from the checkerboard,
// x <- x / |x|, y = M^{-1} K x, lam = |y|, x <- y.
biot_status power_method(biot_ctx* ctx, GmgLevel& L) {
  const int N = 2 * L.nn;
  double *x = nullptr, *y = nullptr, *part = nullptr;
  BIOT_TRY(dalloc(ctx, (void**)&x, sizeof(double) * N));
  BIOT_TRY(dalloc(ctx, (void**)&y, sizeof(double) * N));
  BIOT_TRY(dalloc(ctx, (void**)&part, sizeof(double) * (kRedBlocks + 2)));
  for (int blk = 0; blk < 2; ++blk) {
    const int Nb = blk == 0 ? 2 * L.nn : L.nn;
    const int g = grid_for(Nb);
    BIOT_LAUNCH(k_gmg_checker, g, kThreads, 0, ctx->stream, L.n, blk, x);
    double lam = 0.0;
    for (int it = 0; it < kPowerIters; ++it) {
      BIOT_TRY(norm_dev(ctx, x, Nb, part, part + kRedBlocks, nullptr));
      BIOT_LAUNCH(k_gmg_div, g, kThreads, 0, ctx->stream, x, Nb, part + kRedBlocks);
      BIOT_LAUNCH(k_gmg_power_apply, grid_for(L.nn), kThreads, 0, ctx->stream, L.n, blk, L.coef64, x, y);
      BIOT_TRY(norm_dev(ctx, y, Nb, part, part + kRedBlocks + 1, &lam));
      std::swap(x, y);
    }
    if (!(lam > 0.0) || !std::isfinite(lam))
      return fail(ctx, BIOT_E_CUDA, "multigrid: power method on level n = %d gave %g", L.n, lam);
    L.lam[blk] = lam;
  }
  BIOT_CU(ctx, cudaGetLastError());
  dfree(ctx, x);
  dfree(ctx, y);
  dfree(ctx, part);
  return BIOT_OK;
}

// Chebyshev coefficients on [lam / 8, 1.1 lam] (step 0: c1 = 0, c2 = 1 / theta; step k:
// rho_k = 1 / (2 sigma - rho_{k-1}), c1 = rho_k rho_{k-1}, c2 = 2 rho_k / delta).
void chebyshev_coefs(GmgLevel& L, int steps) {
  for (int blk = 0; blk < 2; ++blk) {
    const double hi = 1.1 * L.lam[blk], lo = L.lam[blk] / kChebLowDiv;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    L.c1[blk][0] = 0.0;
    L.c2[blk][0] = 1.0 / theta;
    for (int k = 1; k < steps; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      L.c1[blk][k] = rn * rho;
      L.c2[blk][k] = 2.0 * rn / delta;
      rho = rn;
    }
  }
}

biot_status level_stencil(biot_ctx* ctx, GmgLevel& L, bool fp64) {
  biot_ctx* o = owner(ctx, L);
  BIOT_TRY(dalloc(o, (void**)&L.coef64, sizeof(double) * (size_t)L.nn * kCoef));
  BIOT_LAUNCH(k_gmg_stencil, grid_for(L.nn), kThreads, 0, ctx->stream, L.n, o->nodeptr, o->nbr, o->rowptr, o->val,
              L.coef64);
  if (!fp64) {
    BIOT_TRY(dalloc(o, (void**)&L.coef32, sizeof(float) * (size_t)L.nn * kCoef));
    BIOT_LAUNCH(k_gmg_to_f32, 512, kThreads, 0, ctx->stream, L.coef64, L.coef32, (size_t)L.nn * kCoef);
  }
  L.dmask = o->dmask;
  BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

biot_status level_buffers(biot_ctx* ctx, GmgLevel& L, int ldg, bool fp64, bool with_e) {
  biot_ctx* o = owner(ctx, L);
  const size_t bytes = (fp64 ? sizeof(double) : sizeof(float)) * (size_t)3 * L.nn * ldg;
  for (int k = 0; k < kGmgBufs; ++k) {
    if (k == GB_E && !with_e) continue;
    BIOT_TRY(dalloc(o, &L.buf[k], bytes));
    BIOT_CU(ctx, cudaMemsetAsync(L.buf[k], 0, bytes, ctx->stream));
  }
  return BIOT_OK;
}

// ---- the cycle (all launches on the fine context's stream) ----

// The level-0 cycle's last smoothing step writes the preconditioner's output z directly.
struct OutZ {
  void* z = nullptr;
  int ld = 0, c0 = 0, ncols = 0;
};

template <typename T, int FM>
void smooth_step(const Gmg& g, GmgLevel& L, cudaStream_t s, int k, bool zero, const T* xin, const T* b, T* xout,
                 const OutZ* oz = nullptr, bool d_from_x = false) {
  constexpr int VEC = V16<T>::n;
  const T cu1 = (T)L.c1[0][k], cu2 = (T)L.c2[0][k], cp1 = (T)L.c1[1][k], cp2 = (T)L.c2[1][k];
  const int nch = g.ldg / VEC;  // every column chunk of the level buffers: unused columns stay finite
  const int grid = grid_stencil((long long)L.nn * nch);
  T* d = buf_of<T>(L, GB_D);
  // the increment is read only by the next step of the same smoothing (k + 1 < smooth); a step
  // from zero leaves it in x, where the next step reads it
  const bool keep_d = !zero && k + 1 < g.smooth;
#define BIOT_SMOOTH(ZERO, READD, OUTZ, DMODE, ...)                                                                \
  BIOT_LAUNCH((k_gmg_smooth<T, FM, ZERO, READD, OUTZ, DMODE>), grid, kThreads, 0, s, L.n, coef_of<T>(L), L.dmask, \
              xin, b, d, __VA_ARGS__)
  if (oz) {  // never the first step of a cycle (k >= 1 or a post-smoothing step): the last one
    T* z = static_cast<T*>(oz->z);
    if (k == 0)
      BIOT_SMOOTH(false, false, true, DM_NO_STORE, z, cu1, cu2, cp1, cp2, g.ldg, 0, nch, oz->ld, oz->c0, oz->ncols);
    else if (d_from_x)
      BIOT_SMOOTH(false, true, true, DM_NO_STORE | DM_FROM_X, z, cu1, cu2, cp1, cp2, g.ldg, 0, nch, oz->ld, oz->c0,
                  oz->ncols);
    else
      BIOT_SMOOTH(false, true, true, DM_NO_STORE, z, cu1, cu2, cp1, cp2, g.ldg, 0, nch, oz->ld, oz->c0, oz->ncols);
    return;
  }
  if (zero)
    BIOT_SMOOTH(true, false, false, DM_NO_STORE, xout, cu1, cu2, cp1, cp2, g.ldg, 0, nch);
  else if (k == 0 && keep_d)
    BIOT_SMOOTH(false, false, false, 0, xout, cu1, cu2, cp1, cp2, g.ldg, 0, nch);
  else if (k == 0)
    BIOT_SMOOTH(false, false, false, DM_NO_STORE, xout, cu1, cu2, cp1, cp2, g.ldg, 0, nch);
  else if (d_from_x && keep_d)
    BIOT_SMOOTH(false, true, false, DM_FROM_X, xout, cu1, cu2, cp1, cp2, g.ldg, 0, nch);
  else if (d_from_x)
    BIOT_SMOOTH(false, true, false, DM_FROM_X | DM_NO_STORE, xout, cu1, cu2, cp1, cp2, g.ldg, 0, nch);
  else if (keep_d)
    BIOT_SMOOTH(false, true, false, 0, xout, cu1, cu2, cp1, cp2, g.ldg, 0, nch);
  else
    BIOT_SMOOTH(false, true, false, DM_NO_STORE, xout, cu1, cu2, cp1, cp2, g.ldg, 0, nch);
#undef BIOT_SMOOTH
}

// One V-cycle on level l for the fields FM: x_out ~ K_l^{-1} b.
template <typename T, int FM>
void vcycle(Gmg& g, int l, cudaStream_t s, const T* b, T* xout, int c0, int ncols, const OutZ* oz = nullptr) {
  constexpr int VEC = V16<T>::n;
  GmgLevel& L = g.lv[l];
  const int nch = g.ldg / VEC;
  if (l == g.L - 1) {
    // exact solve by the level context's band factors (its P2 apply on vin = +-b d)
    T* vin = buf_of<T>(L, GB_R);
    BIOT_LAUNCH((k_gmg_coarse_prep<T, FM>), grid_for((long long)L.nn * ncols), kThreads, 0, s, L.nn, b, L.lc->dsc,
                vin, g.ldg, c0, ncols);
    precond_apply<T>(L.lc, vin, xout, c0, ncols);
    return;
  }
  GmgLevel& C = g.lv[l + 1];
  T* xa = buf_of<T>(L, GB_XA);
  T* xb = buf_of<T>(L, GB_XB);
  // pre-smoothing from zero
  smooth_step<T, FM>(g, L, s, 0, true, nullptr, b, xa);
  for (int k = 1; k < g.smooth; ++k) {
    smooth_step<T, FM>(g, L, s, k, false, xa, b, xb, nullptr, k == 1);
    std::swap(xa, xb);
  }
  // coarse-grid correction
  T* r = buf_of<T>(L, GB_R);
  BIOT_LAUNCH((k_gmg_residual<T, FM>), grid_stencil((long long)L.nn * nch), kThreads, 0, s, L.n, coef_of<T>(L), xa, b,
              r, g.ldg, 0, nch);
  BIOT_LAUNCH((k_gmg_restrict<T, FM>), grid_stencil((long long)C.nn * nch), kThreads, 0, s, C.n, r, C.dmask,
              buf_of<T>(C, GB_B), g.ldg, 0, nch);
  vcycle<T, FM>(g, l + 1, s, buf_of<T>(C, GB_B), buf_of<T>(C, GB_X), c0, ncols);
  BIOT_LAUNCH((k_gmg_prolong<T, FM>), grid_for((long long)L.nn * nch), kThreads, 0, s, L.n, buf_of<T>(C, GB_X), xa,
              g.ldg, 0, nch);
  // post-smoothing: the last step writes x_out
  for (int k = 0; k < g.smooth; ++k) {
    const bool last = k == g.smooth - 1;
    smooth_step<T, FM>(g, L, s, k, false, xa, b, last ? xout : xb, last ? oz : nullptr);
    std::swap(xa, xb);
  }
}

// `cycles` V-cycles on level 0 from zero: x <- V(b); x <- x + V(b - K x).
// Returns true when the result went straight into oz (one cycle), false when it is in the X buffer.
template <typename T, int FM>
bool solve_level0(Gmg& g, cudaStream_t s, int c0, int ncols, const OutZ* oz) {
  constexpr int VEC = V16<T>::n;
  GmgLevel& L = g.lv[0];
  const int nch = g.ldg / VEC;
  T* b = buf_of<T>(L, GB_B);
  T* x = buf_of<T>(L, GB_X);
  if (g.cycles == 1 && g.L > 1) {
    vcycle<T, FM>(g, 0, s, b, x, c0, ncols, oz);
    return true;
  }
  vcycle<T, FM>(g, 0, s, b, x, c0, ncols);
  for (int k = 1; k < g.cycles; ++k) {
    // e = b - K x; correction V(e) into the R buffer (the cycle's own residual there is
    // consumed by its restriction before its last smoothing step writes the correction)
    T* e = buf_of<T>(L, GB_E);
    T* corr = buf_of<T>(L, GB_R);
    BIOT_LAUNCH((k_gmg_residual<T, FM>), grid_stencil((long long)L.nn * nch), kThreads, 0, s, L.n, coef_of<T>(L), x, b,
                e, g.ldg, 0, nch);
    vcycle<T, FM>(g, 0, s, e, corr, c0, ncols);
    BIOT_LAUNCH((k_gmg_axpy<T, FM>), grid_for((long long)L.nn * nch), kThreads, 0, s, L.nn, corr, x, g.ldg, 0, nch);
  }
  return false;
}

template <typename T> T* gmg_tp(biot_ctx* ctx);
template <> double* gmg_tp<double>(biot_ctx* ctx) { return ctx->tp; }
template <> float* gmg_tp<float>(biot_ctx* ctx) { return ctx->lp.tp; }

}  // namespace

// ---- entry points used by the rest of the library ----

void gmg_free(biot_ctx* ctx) {
  Gmg* g = ctx->gmg;
  if (!g) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (GmgLevel& L : g->lv) {
    if (L.lc) {
      biot_destroy(L.lc);  // frees the level's buffers (allocated on it)
      L.lc = nullptr;
    } else {
      for (int k = 0; k < kGmgBufs; ++k) dfree(ctx, L.buf[k]);
      dfree(ctx, L.coef64);
      dfree(ctx, L.coef32);
    }
  }
  delete g;
  ctx->gmg = nullptr;
}

// Levels for an n x n mesh: req <= 0 coarsens while n is even and above kMinCoarse; req >= 2
// asks for that many levels, coarsening while n is even and the coarse mesh keeps two cells.
int gmg_levels_for(int n, int req) {
  int L = 1, m = n;
  if (req <= 0) {
    while (m % 2 == 0 && m > kMinCoarse) {
      m /= 2;
      ++L;
    }
  } else {
    while (m % 2 == 0 && m / 2 >= 2 && L < req) {
      m /= 2;
      ++L;
    }
  }
  return L;
}

biot_status gmg_setup(biot_ctx* ctx) {
  gmg_free(ctx);
  const int L = gmg_levels_for(ctx->n, ctx->gmg_levels_req);
  if (L < 2) return fail(ctx, BIOT_E_INVALID, "multigrid: n = %d cannot be coarsened", ctx->n);
  if (ctx->gmg_smooth < 1 || ctx->gmg_smooth > kMaxSmooth)
    return fail(ctx, BIOT_E_INVALID, "smoothing steps %d outside 1..%d", ctx->gmg_smooth, kMaxSmooth);
  Gmg* g = new Gmg();
  ctx->gmg = g;
  g->L = L;
  g->cycles = ctx->gmg_cycles;
  g->smooth = ctx->gmg_smooth;
  g->ldg = (ctx->wcap + 3) & ~3;
  if ((long long)ctx->n_nodes * (g->ldg / 2) >= (1LL << 31))  // 32-bit work indices of the level-0 kernels
    return fail(ctx, BIOT_E_INVALID, "multigrid: mesh x window too large (%d nodes x %d columns)", ctx->n_nodes,
                g->ldg);
  g->fp64 = ctx->prm.precision == BIOT_FP64;
  g->lv.resize(L);
  double* kprev = ctx->kappa;
  for (int l = 0; l < L; ++l) {
    GmgLevel& Lv = g->lv[l];
    Lv.n = ctx->n >> l;
    Lv.nn = (Lv.n + 1) * (Lv.n + 1);
    if (l > 0) {
      // coarse permeability (mean of the four children) on the device, then assemble the level
      const int nc = Lv.n;
      double* kc = nullptr;
      BIOT_TRY(dalloc(ctx, (void**)&kc, sizeof(double) * 2 * (size_t)nc * nc));
      BIOT_LAUNCH(k_gmg_coarsen_kappa, grid_for(2LL * nc * nc), kThreads, 0, ctx->stream, 2 * nc, kprev, kc);
      std::vector<double> kh(2 * (size_t)nc * nc);
      BIOT_CU(ctx, cudaMemcpyAsync(kh.data(), kc, sizeof(double) * kh.size(), cudaMemcpyDeviceToHost, ctx->stream));
      BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
      dfree(ctx, kc);
      biot_ctx* lc = nullptr;
      biot_status st = biot_mesh_create(nc, ctx->Lx, ctx->Ly, ctx->stream, &lc);
      if (st != BIOT_OK) return fail(ctx, st, "multigrid level n = %d: %s", nc, biot_last_error(nullptr));
      Lv.lc = lc;
      lc->beta_force = ctx->beta;  // the fine level's beta (Galerkin coarse operator)
      lc->sub_req = 1;             // the coarsest level solves by plain band factors
      biot_params p = ctx->prm;
      p.kappa_elem = kh.data();
      p.n_t = l == L - 1 ? g->ldg : 1;  // the coarsest level's band solves take every column
      p.window = 0;
      p.n_iter = 1;
      p.schedule = BIOT_SCHED_TOL;
      st = biot_assemble(lc, &p);
      if (st != BIOT_OK) return fail(ctx, st, "multigrid level n = %d: %s", nc, biot_last_error(lc));
      if (l == L - 1) {
        st = biot_precond_setup(lc, BIOT_PRECOND_DIAG);
        if (st != BIOT_OK) return fail(ctx, st, "multigrid coarsest level n = %d: %s", nc, biot_last_error(lc));
      }
      kprev = lc->kappa;
    }
    BIOT_TRY(level_stencil(ctx, Lv, g->fp64));
    BIOT_TRY(level_buffers(ctx, Lv, g->ldg, g->fp64, l == 0 && g->cycles > 1));
    BIOT_TRY(power_method(ctx, Lv));
    chebyshev_coefs(Lv, g->smooth);
  }
  BIOT_CU(ctx, cudaStreamSynchronize(ctx->stream));
  return BIOT_OK;
}

// z = P^{-1} (vin ./ d) with the block solves replaced by V-cycles (columns [c0, c0 + ncols)).
template <typename T>
void gmg_apply(biot_ctx* ctx, const T* vin, T* z, int c0, int ncols) {
  Gmg& g = *ctx->gmg;
  GmgLevel& L0 = g.lv[0];
  cudaStream_t s = ctx->stream;
  const int nn = ctx->n_nodes, ld = ctx->wcap;
  const int ge = grid_for((long long)nn * ncols);
  const int gp = grid_for((long long)nn * (g.ldg / V16<T>::n));
  T* b = buf_of<T>(L0, GB_B);
  T* x = buf_of<T>(L0, GB_X);
  OutZ oz;
  oz.z = z;
  oz.ld = ld;
  oz.c0 = c0;
  oz.ncols = ncols;
  if (ctx->precond == BIOT_PRECOND_DIAG) {
    BIOT_LAUNCH(k_gmg_prep<T>, gp, kThreads, 0, s, nn, 3, vin, ctx->dsq, (const T*)nullptr, b, ld, g.ldg, c0, ncols);
    if (!solve_level0<T, 3>(g, s, c0, ncols, &oz))
      BIOT_LAUNCH((k_gmg_finish<T, 3>), ge, kThreads, 0, s, nn, x, z, ld, g.ldg, c0, ncols);
  } else {
    BIOT_LAUNCH(k_gmg_prep<T>, gp, kThreads, 0, s, nn, 0, vin, ctx->dsq, (const T*)nullptr, b, ld, g.ldg, c0, ncols);
    if (!solve_level0<T, 1>(g, s, c0, ncols, &oz))
      BIOT_LAUNCH((k_gmg_finish<T, 1>), ge, kThreads, 0, s, nn, x, z, ld, g.ldg, c0, ncols);
    T* tp = gmg_tp<T>(ctx);
    launch_coupling<T>(ctx, z, vin, tp, c0, ncols);  // tp = B^T z_u - vin_p / d
    BIOT_LAUNCH(k_gmg_prep<T>, gp, kThreads, 0, s, nn, 2, (const T*)nullptr, ctx->dsq, tp, b, ld, g.ldg, c0, ncols);
    if (!solve_level0<T, 2>(g, s, c0, ncols, &oz))
      BIOT_LAUNCH((k_gmg_finish<T, 2>), ge, kThreads, 0, s, nn, x, z, ld, g.ldg, c0, ncols);
  }
}
template void gmg_apply<double>(biot_ctx*, const double*, double*, int, int);
template void gmg_apply<float>(biot_ctx*, const float*, float*, int, int);

// ---- batched form: every instance's V-cycle in the same launches (blockIdx.z = instance) ----

namespace {

// One (instance, level) of a batch, as the batched kernels see it.
struct GmgLvDev {
  int active;       // the level smooths and restricts (l < L_i - 1)
  int cl;           // the instance's coarsest level L_i - 1 (the same in every entry of the instance)
  int n, nn, ldg;
  const float* coef;
  const uint8_t* dmask;
  const double* dsc;  // the level context's d (the coarsest level's input scaling)
  float* buf[kGmgBufs];
  float c1[2][kMaxSmooth], c2[2][kMaxSmooth];
};

__device__ __forceinline__ bool batch_live(const InstDev& I) { return I.active && I.nf > 0; }

__global__ void __launch_bounds__(kThreads)
kb_gmg_prep(const InstDev* __restrict__ tab, const GmgLvDev* __restrict__ gt, int Lmax, int j, int mode) {
  const InstDev& I = tab[blockIdx.z];
  if (!batch_live(I)) return;
  const GmgLvDev& e = gt[blockIdx.z * Lmax];
  const size_t vs = (size_t)I.n_dof * I.wcap;
  prep_body<float>(e.nn, mode, I.V + (size_t)j * vs, I.dsq, I.tp, e.buf[GB_B], I.wcap, e.ldg, I.c0, I.nf);
}

// in < 0: from zero; OUTZ: the result goes to the instance's Z_j (level 0, last step).
template <int FM, bool ZERO, bool READD, bool OUTZ>
__global__ void __launch_bounds__(kThreads)
kb_gmg_smooth(const InstDev* __restrict__ tab, const GmgLvDev* __restrict__ gt, int Lmax, int l, int k, int in,
              int out, int j) {
  const InstDev& I = tab[blockIdx.z];
  if (!batch_live(I)) return;
  const GmgLvDev& e = gt[blockIdx.z * Lmax + l];
  if (!e.active) return;
  const int nch = e.ldg / 4;
  float* z = OUTZ ? I.Z + (size_t)j * I.n_dof * I.wcap : e.buf[out];
  smooth_body<float, FM, ZERO, READD, OUTZ>(e.n, e.coef, e.dmask, in < 0 ? nullptr : e.buf[in], e.buf[GB_B],
                                            e.buf[GB_D], z, e.c1[0][k], e.c2[0][k], e.c1[1][k], e.c2[1][k], e.ldg,
                                            0, nch, I.wcap, I.c0, I.nf);
}

template <int FM>
__global__ void __launch_bounds__(kThreads)
kb_gmg_residual_restrict(const InstDev* __restrict__ tab, const GmgLvDev* __restrict__ gt, int Lmax, int l, int in,
                         int phase) {
  const InstDev& I = tab[blockIdx.z];
  if (!batch_live(I)) return;
  const GmgLvDev& e = gt[blockIdx.z * Lmax + l];
  if (!e.active) return;
  const int nch = e.ldg / 4;
  if (phase == 0) {
    residual_body<float, FM>(e.n, e.coef, e.buf[in], e.buf[GB_B], e.buf[GB_R], e.ldg, 0, nch);
  } else {
    const GmgLvDev& c = gt[blockIdx.z * Lmax + l + 1];
    restrict_body<float, FM>(c.n, e.buf[GB_R], c.dmask, c.buf[GB_B], e.ldg, 0, nch);
  }
}

template <int FM>
__global__ void __launch_bounds__(kThreads)
kb_gmg_prolong(const InstDev* __restrict__ tab, const GmgLvDev* __restrict__ gt, int Lmax, int l, int cur) {
  const InstDev& I = tab[blockIdx.z];
  if (!batch_live(I)) return;
  const GmgLvDev& e = gt[blockIdx.z * Lmax + l];
  if (!e.active) return;
  const GmgLvDev& c = gt[blockIdx.z * Lmax + l + 1];
  prolong_body<float, FM>(e.n, c.buf[GB_X], e.buf[cur], e.ldg, 0, e.ldg / 4);
}

template <int FM>
__global__ void kb_gmg_coarse_prep(const InstDev* __restrict__ tab, const GmgLvDev* __restrict__ gt, int Lmax) {
  const InstDev& I = tab[blockIdx.z];
  if (!batch_live(I)) return;
  const GmgLvDev& e = gt[blockIdx.z * Lmax + gt[blockIdx.z * Lmax].cl];
  coarse_prep_body<float, FM>(e.nn, e.buf[GB_B], e.dsc, e.buf[GB_R], e.ldg, I.c0, I.nf);
}

}  // namespace

struct GmgBatch {
  int count = 0, Lmax = 0, smooth = 2, max_band_c = 0, max_wcap_c = 0;
  std::vector<long long> work;  // per level: the largest nn x (ldg / 4) over the instances
  GmgLvDev* gt_d = nullptr;
  InstDev* ct_d = nullptr;      // the coarsest levels' contexts, as batched band-solve instances
  std::vector<InstDev> ct_h;
};

bool gmg_batchable(const biot_ctx* c, const biot_ctx* c0) {
  return c->gmg && c0->gmg && c->gmg->cycles == 1 && c->gmg->smooth == c0->gmg->smooth && !c->gmg->fp64;
}

biot_status gmg_batch_create(biot_ctx* const* ctxs, int count, cudaStream_t s, GmgBatch** out) {
  GmgBatch* gb = new GmgBatch();
  gb->count = count;
  gb->smooth = ctxs[0]->gmg->smooth;
  for (int i = 0; i < count; ++i) gb->Lmax = std::max(gb->Lmax, ctxs[i]->gmg->L);
  gb->work.assign(gb->Lmax, 0);
  std::vector<GmgLvDev> gt((size_t)count * gb->Lmax);
  gb->ct_h.resize(count);
  for (int i = 0; i < count; ++i) {
    Gmg& g = *ctxs[i]->gmg;
    for (int l = 0; l < gb->Lmax; ++l) {
      GmgLvDev& e = gt[(size_t)i * gb->Lmax + l];
      std::memset(&e, 0, sizeof(e));
      e.cl = g.L - 1;
      if (l >= g.L) continue;
      GmgLevel& L = g.lv[l];
      e.active = l < g.L - 1;
      e.n = L.n;
      e.nn = L.nn;
      e.ldg = g.ldg;
      e.coef = L.coef32;
      e.dmask = L.dmask;
      e.dsc = L.lc ? L.lc->dsc : ctxs[i]->dsc;
      for (int k = 0; k < kGmgBufs; ++k) e.buf[k] = static_cast<float*>(L.buf[k]);
      for (int b = 0; b < 2; ++b)
        for (int k = 0; k < kMaxSmooth; ++k) {
          e.c1[b][k] = (float)L.c1[b][k];
          e.c2[b][k] = (float)L.c2[b][k];
        }
      gb->work[l] = std::max(gb->work[l], (long long)L.nn * (g.ldg / 4));
    }
    GmgLevel& C = g.lv[g.L - 1];
    biot_ctx* lc = C.lc;
    BIOT_TRY(ensure_batch_dnb(lc));
    InstDev I = inst_describe(lc);
    I.V = static_cast<float*>(C.buf[GB_R]);  // the coarsest level's input, then its band solves
    I.Z = static_cast<float*>(C.buf[GB_X]);
    gb->ct_h[i] = I;
    gb->max_band_c = std::max(gb->max_band_c, std::max(lc->band_u, lc->band_p));
    gb->max_wcap_c = std::max(gb->max_wcap_c, lc->wcap);
  }
  biot_ctx* c0 = ctxs[0];
  cudaError_t e = cudaMalloc(&gb->gt_d, sizeof(GmgLvDev) * gt.size());
  if (e == cudaSuccess) e = cudaMalloc(&gb->ct_d, sizeof(InstDev) * count);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(gb->gt_d, gt.data(), sizeof(GmgLvDev) * gt.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    gmg_batch_free(gb);
    return fail(c0, BIOT_E_CUDA, "batched multigrid tables: %s", cudaGetErrorString(e));
  }
  *out = gb;
  return BIOT_OK;
}

cudaError_t gmg_batch_update(GmgBatch* gb, const InstDev* tab_h, cudaStream_t s) {
  for (int i = 0; i < gb->count; ++i) {
    gb->ct_h[i].active = tab_h[i].active;
    gb->ct_h[i].c0 = tab_h[i].c0;
    gb->ct_h[i].nf = tab_h[i].nf;
  }
  return cudaMemcpyAsync(gb->ct_d, gb->ct_h.data(), sizeof(InstDev) * gb->count, cudaMemcpyHostToDevice, s);
}

namespace {

template <int FM>
void batch_vcycle(GmgBatch* gb, const InstDev* tab, int count, int j, cudaStream_t s) {
  const int Lm = gb->Lmax, m = gb->smooth;
  const GmgLvDev* gt = gb->gt_d;
  // the buffer holding a level's iterate after its pre-smoothing (the same for every level)
  int cur = GB_XA;
  for (int l = 0; l + 1 < Lm; ++l) {
    const dim3 grid(grid_stencil(gb->work[l]), 1, count);
    BIOT_LAUNCH((kb_gmg_smooth<FM, true, false, false>), grid, kThreads, 0, s, tab, gt, Lm, l, 0, -1, GB_XA, j);
    cur = GB_XA;
    for (int k = 1; k < m; ++k) {
      const int nxt = cur == GB_XA ? GB_XB : GB_XA;
      BIOT_LAUNCH((kb_gmg_smooth<FM, false, true, false>), grid, kThreads, 0, s, tab, gt, Lm, l, k, cur, nxt, j);
      cur = nxt;
    }
    BIOT_LAUNCH((kb_gmg_residual_restrict<FM>), grid, kThreads, 0, s, tab, gt, Lm, l, cur, 0);
    BIOT_LAUNCH((kb_gmg_residual_restrict<FM>), dim3(grid_stencil(gb->work[l + 1]), 1, count), kThreads, 0, s, tab, gt,
                Lm, l, cur, 1);
  }
  // every instance's coarsest level at once: +-b d, then the batched exact P2 band solves
  BIOT_LAUNCH((kb_gmg_coarse_prep<FM>), dim3(64, 1, count), kThreads, 0, s, tab, gt, Lm);
  batched_precond_apply(gb->ct_d, count, 0, gb->max_wcap_c, gb->max_band_c, false, s);
  for (int l = Lm - 2; l >= 0; --l) {
    const dim3 grid(grid_for(gb->work[l]), 1, count);
    int c = cur;
    BIOT_LAUNCH((kb_gmg_prolong<FM>), grid, kThreads, 0, s, tab, gt, Lm, l, c);
    for (int k = 0; k < m; ++k) {
      const bool last = k == m - 1;
      const int nxt = c == GB_XA ? GB_XB : GB_XA;
      if (last && l == 0) {
        if (k == 0) BIOT_LAUNCH((kb_gmg_smooth<FM, false, false, true>), grid, kThreads, 0, s, tab, gt, Lm, l, k, c, 0, j);
        else BIOT_LAUNCH((kb_gmg_smooth<FM, false, true, true>), grid, kThreads, 0, s, tab, gt, Lm, l, k, c, 0, j);
      } else {
        const int dst = last ? GB_X : nxt;
        if (k == 0) BIOT_LAUNCH((kb_gmg_smooth<FM, false, false, false>), grid, kThreads, 0, s, tab, gt, Lm, l, k, c, dst, j);
        else BIOT_LAUNCH((kb_gmg_smooth<FM, false, true, false>), grid, kThreads, 0, s, tab, gt, Lm, l, k, c, dst, j);
        c = dst;
      }
    }
  }
}

}  // namespace

void gmg_batch_apply(GmgBatch* gb, const InstDev* tab, int count, int j, bool tri, cudaStream_t s) {
  const GmgLvDev* gt = gb->gt_d;
  const dim3 g0(grid_for(gb->work[0]), 1, count);
  if (!tri) {
    BIOT_LAUNCH(kb_gmg_prep, g0, kThreads, 0, s, tab, gt, gb->Lmax, j, 3);
    batch_vcycle<3>(gb, tab, count, j, s);
  } else {
    BIOT_LAUNCH(kb_gmg_prep, g0, kThreads, 0, s, tab, gt, gb->Lmax, j, 0);
    batch_vcycle<1>(gb, tab, count, j, s);
    launch_batched_coupling(tab, count, j, s);  // tp = B^T z_u - v_p / d per instance
    BIOT_LAUNCH(kb_gmg_prep, g0, kThreads, 0, s, tab, gt, gb->Lmax, j, 2);
    batch_vcycle<2>(gb, tab, count, j, s);
  }
}

void gmg_batch_free(GmgBatch* gb) {
  if (!gb) return;
  if (gb->gt_d) cudaFree(gb->gt_d);
  if (gb->ct_d) cudaFree(gb->ct_d);
  delete gb;
}

void gmg_info(const biot_ctx* ctx, int* levels, double* lam_u, double* lam_p) {
  const Gmg* g = ctx->gmg;
  *levels = g ? g->L : 0;
  *lam_u = g ? g->lv[0].lam[0] : 0.0;
  *lam_p = g ? g->lv[0].lam[1] : 0.0;
}

}  // namespace biot
