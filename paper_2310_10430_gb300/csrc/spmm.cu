// Multi-right-hand-side sparse products of the sweep.
//
// The residual of every active time step (Alg. 3: b^{n,m} = A' X^{n-1,m} + f^n,
// r = b - AA X^{n,m-1}) is formed in one pass over the matrix: a warp owns one
// mesh node (three CSR rows: u_x, u_y, p) and its lanes own consecutive time
// steps. The state X is stored [DOF][time] (time fastest), so a warp's loads of
// X[dof][lo-1 .. hi] are contiguous. Each 3x3 node block of AA is read once per
// node and applied to all active steps; A' shares B^T with AA and adds its own
// pressure-pressure entry, applied to X at step n-1.
//
// Types: XT is the vector type (double for the FP64 path, float for the
// reduced-precision sweep), VT the stored matrix-value type (double, float or
// __nv_bfloat16); products accumulate in XT; norms are combined in FP64 across
// lanes and blocks.
#include "common.cuh"

#include <algorithm>
#include <cstdio>
#include <map>
#include <string>

namespace biot {

namespace {

constexpr int kWarps = 8;

template <typename T> __device__ __forceinline__ T ld_val(const T* p) { return *p; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }

template <typename XT> struct Acc;
template <> struct Acc<double> { using T = double; };
template <> struct Acc<float> { using T = float; };

// Reduce one double per (warp, lane) over the block's warps in warp order and
// store it at dst[lane] for lanes < count (called by all threads).
__device__ __forceinline__ void block_sum_to(double (*sm)[32], double val, double* dst, int count) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  sm[warp][lane] = val;
  __syncthreads();
  if (warp == 0) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += sm[w][lane];
    if (lane < count) dst[lane] = s;
  }
  __syncthreads();
}

// out[3v+f][c] = (EQ ? d : 1) * (F + A' X_{n-1} - AA X_n)[3v+f], n = lo + c; partial |d r|^2 and
// |d b|^2 in part slots 0 and 1.
template <typename XT, typename VT, typename OT, bool EQ>
__device__ __forceinline__ void residual_body(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
           const int32_t* __restrict__ rowptr, const VT* __restrict__ val, const VT* __restrict__ apval,
           const double* __restrict__ dsc, const XT* __restrict__ X, const XT* __restrict__ F, int ldx, int lo,
           int ncols, OT* __restrict__ out, int ldo, int ocol0, double* __restrict__ part, int ldp) {
  using A = typename Acc<XT>::T;
  __shared__ double sm[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nn + gridDim.x - 1) / gridDim.x;
  const int vb = blockIdx.x * per, ve = min(nn, vb + per);
  for (int cb = 0; cb < ncols; cb += 32) {
    const int c = cb + lane;
    const bool cv = c < ncols;
    const int tn = lo + (cv ? c : 0);  // time step of this lane
    A rr = 0, bb = 0;
    for (int v = vb + warp; v < ve; v += kWarps) {
      const int32_t np = nodeptr[v];
      const int deg = nodeptr[v + 1] - np;
      const int32_t r0 = rowptr[3 * v], r1 = r0 + 3 * deg, r2 = r1 + 3 * deg;
      const A f0 = F[(size_t)(3 * v) * ldx + tn];
      const A f1 = F[(size_t)(3 * v + 1) * ldx + tn];
      const A f2 = F[(size_t)(3 * v + 2) * ldx + tn];
      A a0 = 0, a1 = 0, a2 = 0, ap = 0;
      for (int k = 0; k < deg; ++k) {
        const int m = nbr[np + k];
        const XT* xm = X + (size_t)(3 * m) * ldx + tn;
        const A x0 = xm[0], x1 = xm[ldx], x2 = xm[2 * ldx];
        const A y0 = xm[-1], y1 = xm[ldx - 1], y2 = xm[2 * ldx - 1];
        const VT* e0 = val + r0 + 3 * k;
        const VT* e1 = val + r1 + 3 * k;
        const VT* e2 = val + r2 + 3 * k;
        a0 += (A)to_acc(e0[0]) * x0 + (A)to_acc(e0[1]) * x1 + (A)to_acc(e0[2]) * x2;
        a1 += (A)to_acc(e1[0]) * x0 + (A)to_acc(e1[1]) * x1 + (A)to_acc(e1[2]) * x2;
        const A b0 = to_acc(e2[0]), b1 = to_acc(e2[1]);
        a2 += b0 * x0 + b1 * x1 + (A)to_acc(e2[2]) * x2;
        ap += b0 * y0 + b1 * y1 + (A)to_acc(apval[np + k]) * y2;
      }
      const A d0 = (A)dsc[3 * v], d1 = (A)dsc[3 * v + 1], d2 = (A)dsc[3 * v + 2];
      const A b2 = f2 + ap;
      const A s0 = f0 - a0, s1 = f1 - a1, s2 = b2 - a2;
      const A q0 = d0 * s0, q1 = d1 * s1, q2 = d2 * s2;
      if (cv) {
        const size_t oc = (size_t)ocol0 + c;
        out[(size_t)(3 * v) * ldo + oc] = (OT)(EQ ? q0 : s0);
        out[(size_t)(3 * v + 1) * ldo + oc] = (OT)(EQ ? q1 : s1);
        out[(size_t)(3 * v + 2) * ldo + oc] = (OT)(EQ ? q2 : s2);
        rr += q0 * q0 + q1 * q1 + q2 * q2;
        const A p0 = d0 * f0, p1 = d1 * f1, p2 = d2 * b2;
        bb += p0 * p0 + p1 * p1 + p2 * p2;
      }
    }
    block_sum_to(sm, (double)rr, part + (size_t)(0 * gridDim.x + blockIdx.x) * ldp + cb, min(32, ncols - cb));
    block_sum_to(sm, (double)bb, part + (size_t)(1 * gridDim.x + blockIdx.x) * ldp + cb, min(32, ncols - cb));
  }
}

template <typename XT, typename VT, typename OT, bool EQ>
__global__ void __launch_bounds__(kWarps * 32)
k_residual(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
           const int32_t* __restrict__ rowptr, const VT* __restrict__ val, const VT* __restrict__ apval,
           const double* __restrict__ dsc, const XT* __restrict__ X, const XT* __restrict__ F, int ldx, int lo,
           int ncols, OT* __restrict__ out, int ldo, int ocol0, double* __restrict__ part, int ldp) {
  residual_body<XT, VT, OT, EQ>(nn, nodeptr, nbr, rowptr, val, apval, dsc, X, F, ldx, lo, ncols, out, ldo, ocol0,
                                part, ldp);
}

// w[:, c] = d .* (AA z[:, c]) for c in [c0, c0 + ncols); partial |w|^2 in slot 0.
template <typename XT, typename VT>
__device__ __forceinline__ void spmm_body(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
              const int32_t* __restrict__ rowptr, const VT* __restrict__ val, const double* __restrict__ dsc,
              const XT* __restrict__ z, XT* __restrict__ w, int ld, int c0, int ncols, double* __restrict__ part) {
  using A = typename Acc<XT>::T;
  __shared__ double sm[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nn + gridDim.x - 1) / gridDim.x;
  const int vb = blockIdx.x * per, ve = min(nn, vb + per);
  for (int cb = 0; cb < ncols; cb += 32) {
    const int c = c0 + cb + lane;
    const bool cv = cb + lane < ncols;
    const int cc = cv ? c : c0;
    A ww = 0;
    for (int v = vb + warp; v < ve; v += kWarps) {
      const int32_t np = nodeptr[v];
      const int deg = nodeptr[v + 1] - np;
      const int32_t r0 = rowptr[3 * v], r1 = r0 + 3 * deg, r2 = r1 + 3 * deg;
      A a0 = 0, a1 = 0, a2 = 0;
      for (int k = 0; k < deg; ++k) {
        const int m = nbr[np + k];
        const XT* zm = z + (size_t)(3 * m) * ld + cc;
        const A x0 = zm[0], x1 = zm[ld], x2 = zm[2 * ld];
        const VT* e0 = val + r0 + 3 * k;
        const VT* e1 = val + r1 + 3 * k;
        const VT* e2 = val + r2 + 3 * k;
        a0 += (A)to_acc(e0[0]) * x0 + (A)to_acc(e0[1]) * x1 + (A)to_acc(e0[2]) * x2;
        a1 += (A)to_acc(e1[0]) * x0 + (A)to_acc(e1[1]) * x1 + (A)to_acc(e1[2]) * x2;
        a2 += (A)to_acc(e2[0]) * x0 + (A)to_acc(e2[1]) * x1 + (A)to_acc(e2[2]) * x2;
      }
      const A q0 = (A)dsc[3 * v] * a0, q1 = (A)dsc[3 * v + 1] * a1, q2 = (A)dsc[3 * v + 2] * a2;
      if (cv) {
        w[(size_t)(3 * v) * ld + c] = (XT)q0;
        w[(size_t)(3 * v + 1) * ld + c] = (XT)q1;
        w[(size_t)(3 * v + 2) * ld + c] = (XT)q2;
        ww += q0 * q0 + q1 * q1 + q2 * q2;
      }
    }
    block_sum_to(sm, (double)ww, part + (size_t)blockIdx.x * ld + c0 + cb, min(32, ncols - cb));
  }
}

// 16-byte vector of XT (four floats or two doubles).
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using V = float4;
  static constexpr int n = 4;
  __device__ __forceinline__ static void get(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ __forceinline__ static V make(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <> struct Vec16<double> {
  using V = double2;
  static constexpr int n = 2;
  __device__ __forceinline__ static void get(const V& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ __forceinline__ static V make(const double* o) { return make_double2(o[0], o[1]); }
};

// VEC-wide vector of XT for the tuned SpMM variants (8 or 16 bytes).
template <typename T, int N> struct VecN;
template <> struct VecN<float, 4> : Vec16<float> {};
template <> struct VecN<double, 2> : Vec16<double> {};
template <> struct VecN<float, 2> {
  using V = float2;
  static constexpr int n = 2;
  __device__ __forceinline__ static void get(const V& v, float* o) { o[0] = v.x; o[1] = v.y; }
  __device__ __forceinline__ static V make(const float* o) { return make_float2(o[0], o[1]); }
};

// spmm_body with 16-byte accesses: a lane owns VEC consecutive columns, so every DOF row
// of z is read with one 128-bit load per lane and a warp covers 32 * VEC columns per
// pass. The column range is widened down to a multiple of VEC; lanes mask what lies
// outside [c0, c0 + ncols). Needs ld % VEC == 0 and 16-byte aligned z and w. The sums
// run in the same order as spmm_body, and the per-column norm partials land in the same
// slots part[block * ld + column].
// VEC (columns per lane) and UNR (neighbour-loop unrolling) are tuned per mesh and window
// (biot_tune); the default is the 16-byte form with UNR = 4.
// ILV: the nodes are dealt out to the warps of the grid in turns (warp w of block b takes nodes
// (t gridDim.x + b) kWarps + w, t = 0, 1, ...) instead of a contiguous range per block: the grid
// then works on a band of a few mesh rows at a time, and the neighbour rows of z in the mesh rows
// above and below are still in L2 (with contiguous ranges the whole of z is live at once and
// those rows came back from DRAM: 2.9 reads of z per launch instead of 1.3).
template <typename XT, typename VT, int VEC = Vec16<XT>::n, int UNR = 4, bool ILV = false>
__device__ __forceinline__ void spmm_vec_body(int nn, const int32_t* __restrict__ nodeptr,
              const int32_t* __restrict__ nbr, const int32_t* __restrict__ rowptr, const VT* __restrict__ val,
              const double* __restrict__ dsc, const XT* __restrict__ z, XT* __restrict__ w, int ld, int c0,
              int ncols, double* __restrict__ part) {
  using A = typename Acc<XT>::T;
  using VN = VecN<XT, VEC>;
  using V = typename VN::V;
  __shared__ double sm[kWarps][32 * VEC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nn + gridDim.x - 1) / gridDim.x;
  const int vb = blockIdx.x * per, ve = min(nn, vb + per);
  const int ca = c0 & ~(VEC - 1), ce = c0 + ncols;
  for (int cb = ca; cb < ce; cb += 32 * VEC) {
    const int c = cb + lane * VEC;
    const bool any = c < ce;
    const bool full = c >= c0 && c + VEC <= ce;
    const int cc = any ? c : ca;
    A ww[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) ww[q] = 0;
    for (int v = ILV ? blockIdx.x * kWarps + warp : vb + warp; v < (ILV ? nn : ve);
         v += ILV ? gridDim.x * kWarps : kWarps) {
      const int32_t np = nodeptr[v];
      const int deg = nodeptr[v + 1] - np;
      const int32_t r0 = rowptr[3 * v], r1 = r0 + 3 * deg, r2 = r1 + 3 * deg;
      A a0[VEC], a1[VEC], a2[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) a0[q] = a1[q] = a2[q] = 0;
#pragma unroll UNR
      for (int k = 0; k < deg; ++k) {
        const int m = nbr[np + k];
        const XT* zm = z + (size_t)(3 * m) * ld + cc;
        XT x0[VEC], x1[VEC], x2[VEC];
        VN::get(*reinterpret_cast<const V*>(zm), x0);
        VN::get(*reinterpret_cast<const V*>(zm + ld), x1);
        VN::get(*reinterpret_cast<const V*>(zm + 2 * ld), x2);
        const VT* e0 = val + r0 + 3 * k;
        const VT* e1 = val + r1 + 3 * k;
        const VT* e2 = val + r2 + 3 * k;
        const A m00 = to_acc(e0[0]), m01 = to_acc(e0[1]), m02 = to_acc(e0[2]);
        const A m10 = to_acc(e1[0]), m11 = to_acc(e1[1]), m12 = to_acc(e1[2]);
        const A m20 = to_acc(e2[0]), m21 = to_acc(e2[1]), m22 = to_acc(e2[2]);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          a0[q] += m00 * (A)x0[q] + m01 * (A)x1[q] + m02 * (A)x2[q];
          a1[q] += m10 * (A)x0[q] + m11 * (A)x1[q] + m12 * (A)x2[q];
          a2[q] += m20 * (A)x0[q] + m21 * (A)x1[q] + m22 * (A)x2[q];
        }
      }
      const A d0 = (A)dsc[3 * v], d1 = (A)dsc[3 * v + 1], d2 = (A)dsc[3 * v + 2];
      XT o0[VEC], o1[VEC], o2[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        const A q0 = d0 * a0[q], q1 = d1 * a1[q], q2 = d2 * a2[q];
        o0[q] = (XT)q0;
        o1[q] = (XT)q1;
        o2[q] = (XT)q2;
        const bool in = c + q >= c0 && c + q < ce;
        if (in) ww[q] += q0 * q0 + q1 * q1 + q2 * q2;
      }
      XT* w0 = w + (size_t)(3 * v) * ld + c;
      if (full) {
        *reinterpret_cast<V*>(w0) = VN::make(o0);
        *reinterpret_cast<V*>(w0 + ld) = VN::make(o1);
        *reinterpret_cast<V*>(w0 + 2 * ld) = VN::make(o2);
      } else if (any) {
#pragma unroll
        for (int q = 0; q < VEC; ++q)
          if (c + q >= c0 && c + q < ce) {
            w0[q] = o0[q];
            w0[ld + q] = o1[q];
            w0[2 * ld + q] = o2[q];
          }
      }
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) sm[warp][lane * VEC + q] = (double)ww[q];
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * VEC; t += blockDim.x) {
      double sum = 0.0;
      for (int u = 0; u < kWarps; ++u) sum += sm[u][t];
      const int col = cb + t;
      if (col >= c0 && col < ce) part[(size_t)blockIdx.x * ld + col] = sum;
    }
    __syncthreads();
  }
}

template <typename XT, typename VT, int VEC = Vec16<XT>::n, int UNR = 4, int MINB = 2, bool ILV = false>
__global__ void __launch_bounds__(kWarps * 32, MINB)
k_spmm_vec(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
           const int32_t* __restrict__ rowptr, const VT* __restrict__ val, const double* __restrict__ dsc,
           const XT* __restrict__ z, XT* __restrict__ w, int ld, int c0, int ncols, double* __restrict__ part) {
  spmm_vec_body<XT, VT, VEC, UNR, ILV>(nn, nodeptr, nbr, rowptr, val, dsc, z, w, ld, c0, ncols, part);
}

template <typename XT, typename VT>
__global__ void __launch_bounds__(kWarps * 32)
k_spmm_scaled(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
              const int32_t* __restrict__ rowptr, const VT* __restrict__ val, const double* __restrict__ dsc,
              const XT* __restrict__ z, XT* __restrict__ w, int ld, int c0, int ncols, double* __restrict__ part) {
  spmm_body<XT, VT>(nn, nodeptr, nbr, rowptr, val, dsc, z, w, ld, c0, ncols, part);
}

// P1 coupling: tp[v][c] = (B^T z_u)[v][c] - vin[3v+2][c] / d[3v+2] (grid-stride over (v, c)).
template <typename XT, typename VT>
__device__ __forceinline__ void coupling_body(int nn, const int32_t* __restrict__ nodeptr,
                                              const int32_t* __restrict__ nbr, const int32_t* __restrict__ rowptr,
                                              const VT* __restrict__ val, const double* __restrict__ dsc,
                                              const XT* __restrict__ z, const XT* __restrict__ vin,
                                              XT* __restrict__ tp, int ld, int c0, int ncols) {
  using A = typename Acc<XT>::T;
  const long long total = (long long)nn * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    const int32_t np = nodeptr[v];
    const int deg = nodeptr[v + 1] - np;
    const int32_t r2 = rowptr[3 * v] + 6 * deg;
    A s = 0;
    for (int k = 0; k < deg; ++k) {
      const int m = nbr[np + k];
      s += (A)to_acc(val[r2 + 3 * k]) * (A)z[(size_t)(3 * m) * ld + c] +
           (A)to_acc(val[r2 + 3 * k + 1]) * (A)z[(size_t)(3 * m + 1) * ld + c];
    }
    tp[(size_t)v * ld + c] = (XT)(s - (A)vin[(size_t)(3 * v + 2) * ld + c] / (A)dsc[3 * v + 2]);
  }
}

template <typename XT, typename VT>
__global__ void k_coupling(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
                           const int32_t* __restrict__ rowptr, const VT* __restrict__ val,
                           const double* __restrict__ dsc, const XT* __restrict__ z, const XT* __restrict__ vin,
                           XT* __restrict__ tp, int ld, int c0, int ncols) {
  coupling_body<XT, VT>(nn, nodeptr, nbr, rowptr, val, dsc, z, vin, tp, ld, c0, ncols);
}

// ---- batched variants: instance = blockIdx.z, arguments from the instance table ----

template <typename VT> __device__ __forceinline__ const VT* inst_val(const InstDev& I);
template <> __device__ __forceinline__ const float* inst_val<float>(const InstDev& I) { return I.val; }
template <> __device__ __forceinline__ const __nv_bfloat16* inst_val<__nv_bfloat16>(const InstDev& I) {
  return I.valbf;
}

// True residual in FP64 of the window, columns [0, nres) of the FP32 V_0 (equilibrated).
__global__ void __launch_bounds__(kWarps * 32) kb_residual(const InstDev* __restrict__ tab) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nres <= 0) return;
  residual_body<double, double, float, true>(I.n_nodes, I.nodeptr, I.nbr, I.rowptr, I.val64, I.apval64, I.dsc, I.X64,
                                             I.F64, I.ldx, I.lo, I.nres, I.V, I.wcap, 0, I.part, I.wcap);
}

template <typename VT>
__global__ void __launch_bounds__(kWarps * 32) kb_spmm(const InstDev* __restrict__ tab, int j) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  const size_t vs = (size_t)I.n_dof * I.wcap;
  spmm_body<float, VT>(I.n_nodes, I.nodeptr, I.nbr, I.rowptr, inst_val<VT>(I), I.dsc, I.Z + j * vs, I.Wv, I.wcap,
                       I.c0, I.nf, I.part);
}

__global__ void kb_coupling(const InstDev* __restrict__ tab, int j) {
  const InstDev& I = tab[blockIdx.z];
  if (!I.active || I.nf <= 0) return;
  const size_t vs = (size_t)I.n_dof * I.wcap;
  coupling_body<float, float>(I.n_nodes, I.nodeptr, I.nbr, I.rowptr, I.val, I.dsc, I.Z + j * vs, I.V + j * vs, I.tp,
                              I.wcap, I.c0, I.nf);
}

}  // namespace

// The 16-byte SpMM needs rows of z and w that start on 16-byte boundaries.
template <typename XT>
static bool vec_ok(const biot_ctx* ctx, const XT* z, const XT* w) {
  constexpr int VEC = Vec16<XT>::n;
  return ctx->wcap % VEC == 0 && reinterpret_cast<uintptr_t>(z) % 16 == 0 && reinterpret_cast<uintptr_t>(w) % 16 == 0;
}

void launch_residual_raw(int n_nodes, const int32_t* nodeptr, const int32_t* nbr, const int32_t* rowptr,
                         const double* val, const double* apval, const double* dsc, const double* X,
                         const double* F, int ldx, int lo, int ncols, double* out, int ldo, double* part, int ldp,
                         cudaStream_t stream) {
  BIOT_LAUNCH((k_residual<double, double, double, true>), kRedBlocks, kWarps * 32, 0, stream, n_nodes, nodeptr, nbr,
              rowptr, val, apval, dsc, X, F, ldx, lo, ncols, out, ldo, 0, part, ldp);
}

void launch_residual(biot_ctx* ctx, int lo, int ncols, double* out, int ldo) {
  KTimer tm(ctx, BIOT_KC_RESIDUAL);
  BIOT_LAUNCH((k_residual<double, double, double, true>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes,
              ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->val, ctx->apval, ctx->dsc, ctx->X, ctx->F, ctx->ldx, lo,
              ncols, out, ldo, 0, ctx->part, ctx->wcap);
}

// Reduced-precision sweep: the true residual in FP64, written equilibrated into the
// FP32 V_0 that starts the FP32 Krylov cycle on the correction.
void launch_residual_lp(biot_ctx* ctx, int lo, int ncols) {
  KTimer tm(ctx, BIOT_KC_RESIDUAL);
  BIOT_LAUNCH((k_residual<double, double, float, true>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes,
              ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->val, ctx->apval, ctx->dsc, ctx->X, ctx->F, ctx->ldx, lo,
              ncols, ctx->lp.V, ctx->wcap, 0, ctx->part, ctx->wcap);
}

template <>
void launch_spmm_scaled<double>(biot_ctx* ctx, const double* z, double* w, int c0, int ncols) {
  KTimer tm(ctx, BIOT_KC_SPMM);
  if (vec_ok<double>(ctx, z, w))
    BIOT_LAUNCH((k_spmm_vec<double, double>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr,
                ctx->nbr, ctx->rowptr, ctx->val, ctx->dsc, z, w, ctx->wcap, c0, ncols, ctx->part);
  else
    BIOT_LAUNCH((k_spmm_scaled<double, double>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes,
                ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->val, ctx->dsc, z, w, ctx->wcap, c0, ncols, ctx->part);
}

// Tuned shapes of the FP32 / BF16-value SpMM (biot_tune): columns per lane (16- or 8-byte
// vectors), unrolling of the neighbour loop, CTAs per SM the registers are sized for, the grid
// in multiples of the 152 SMs (also the number of norm partials per column) and whether the
// nodes are dealt out in turns (ilv, shapes 6-7) or in a contiguous range per block.
struct SpmmVariant {
  int vec, unr, minb, gmul, ilv;
};
constexpr SpmmVariant kSpmmVariants[] = {{4, 4, 2, 2, 0}, {4, 2, 3, 3, 0}, {4, 2, 4, 4, 0}, {2, 4, 2, 2, 0},
                                         {2, 2, 4, 4, 0}, {4, 1, 4, 4, 0}, {4, 2, 4, 4, 1}, {4, 1, 4, 4, 1}};
constexpr int kSpmmVariantCount = sizeof(kSpmmVariants) / sizeof(kSpmmVariants[0]);

template <typename VT>
static void launch_spmm_variant(biot_ctx* ctx, int v, const VT* val, const float* z, float* w, int c0, int ncols) {
  const int grid = kSpmmVariants[v].gmul * 152;
#define BIOT_SPMM_CASE(id, VEC, UNR, MINB, ILV)                                                                    \
  case id:                                                                                                          \
    BIOT_LAUNCH((k_spmm_vec<float, VT, VEC, UNR, MINB, ILV>), grid, kWarps * 32, 0, ctx->stream, ctx->n_nodes,     \
                ctx->nodeptr, ctx->nbr, ctx->rowptr, val, ctx->dsc, z, w, ctx->wcap, c0, ncols, ctx->part);         \
    break;
  switch (v) {
    BIOT_SPMM_CASE(1, 4, 2, 3, false)
    BIOT_SPMM_CASE(2, 4, 2, 4, false)
    BIOT_SPMM_CASE(3, 2, 4, 2, false)
    BIOT_SPMM_CASE(4, 2, 2, 4, false)
    BIOT_SPMM_CASE(5, 4, 1, 4, false)
    BIOT_SPMM_CASE(6, 4, 2, 4, true)
    BIOT_SPMM_CASE(7, 4, 1, 4, true)
    default:
      BIOT_LAUNCH((k_spmm_vec<float, VT>), grid, kWarps * 32, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr, ctx->nbr,
                  ctx->rowptr, val, ctx->dsc, z, w, ctx->wcap, c0, ncols, ctx->part);
  }
#undef BIOT_SPMM_CASE
}

static bool spmm_variant_ok(const biot_ctx* ctx, int v, const float* z, const float* w) {
  const int vec = kSpmmVariants[v].vec;
  return ctx->wcap % vec == 0 && reinterpret_cast<uintptr_t>(z) % (4 * vec) == 0 &&
         reinterpret_cast<uintptr_t>(w) % (4 * vec) == 0;
}

// Blocks (norm partials per column) of the SpMM launch_spmm_scaled issues for this context.
int spmm_blocks(const biot_ctx* ctx) {
  if (ctx->prm.precision == BIOT_FP64) return kRedBlocks;
  return kSpmmVariants[ctx->spmm_var].gmul * 152;
}

template <>
void launch_spmm_scaled<float>(biot_ctx* ctx, const float* z, float* w, int c0, int ncols) {
  KTimer tm(ctx, BIOT_KC_SPMM);
  const bool vec = vec_ok<float>(ctx, z, w);
  const int v = ctx->spmm_var;
  if (v != 0 && spmm_variant_ok(ctx, v, z, w)) {
    if (ctx->prm.precision == BIOT_BF16VAL_FP32ACC) launch_spmm_variant(ctx, v, ctx->lp.val_bf16, z, w, c0, ncols);
    else launch_spmm_variant(ctx, v, ctx->lp.val, z, w, c0, ncols);
    return;
  }
  if (ctx->prm.precision == BIOT_BF16VAL_FP32ACC) {
    if (vec)
      BIOT_LAUNCH((k_spmm_vec<float, __nv_bfloat16>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes,
                  ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->lp.val_bf16, ctx->dsc, z, w, ctx->wcap, c0, ncols,
                  ctx->part);
    else
      BIOT_LAUNCH((k_spmm_scaled<float, __nv_bfloat16>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes,
                  ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->lp.val_bf16, ctx->dsc, z, w, ctx->wcap, c0, ncols,
                  ctx->part);
  } else {
    if (vec)
      BIOT_LAUNCH((k_spmm_vec<float, float>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes,
                  ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->lp.val, ctx->dsc, z, w, ctx->wcap, c0, ncols, ctx->part);
    else
      BIOT_LAUNCH((k_spmm_scaled<float, float>), kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes,
                  ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->lp.val, ctx->dsc, z, w, ctx->wcap, c0, ncols, ctx->part);
  }
}

template <>
void launch_coupling<double>(biot_ctx* ctx, const double* z, const double* vin, double* tp, int c0, int ncols) {
  const int grid = std::min(div_up((long long)ctx->n_nodes * ncols, 256), 4096);
  BIOT_LAUNCH((k_coupling<double, double>), grid, 256, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr, ctx->nbr,
              ctx->rowptr, ctx->val, ctx->dsc, z, vin, tp, ctx->wcap, c0, ncols);
}

template <>
void launch_coupling<float>(biot_ctx* ctx, const float* z, const float* vin, float* tp, int c0, int ncols) {
  // the preconditioner's coupling block B^T runs in FP32 in both reduced-precision modes
  const int grid = std::min(div_up((long long)ctx->n_nodes * ncols, 256), 4096);
  BIOT_LAUNCH((k_coupling<float, float>), grid, 256, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr, ctx->nbr,
              ctx->rowptr, ctx->lp.val, ctx->dsc, z, vin, tp, ctx->wcap, c0, ncols);
}

void launch_batched_residual(const InstDev* tab, int count, cudaStream_t s) {
  BIOT_LAUNCH(kb_residual, dim3(kRedBlocks, 1, count), kWarps * 32, 0, s, tab);
}

void launch_batched_spmm(const InstDev* tab, int count, bool bf16, int j, cudaStream_t s) {
  dim3 grid(kRedBlocks, 1, count);
  if (bf16) BIOT_LAUNCH(kb_spmm<__nv_bfloat16>, grid, kWarps * 32, 0, s, tab, j);
  else BIOT_LAUNCH(kb_spmm<float>, grid, kWarps * 32, 0, s, tab, j);
}

void launch_batched_coupling(const InstDev* tab, int count, int j, cudaStream_t s) {
  BIOT_LAUNCH(kb_coupling, dim3(256, 1, count), 256, 0, s, tab, j);
}

// Time every SpMM shape on this context's FP32 (or BF16) values at full window width (w = d .*
// AA z on the first two Krylov vectors; best of three after a warm-up) and keep the fastest;
// cached under "spmm:" + precision, rows and window. Returns the chosen and the default times.
biot_status spmm_tune(biot_ctx* ctx, std::map<std::string, int>* cache, int* hit, double* ms_best,
                      double* ms_default) {
  *hit = 0;
  *ms_best = *ms_default = 0.0;
  if (ctx->prm.precision == BIOT_FP64) return BIOT_OK;
  char key[96];
  snprintf(key, sizeof(key), "spmm:%s:N%d:w%d", ctx->prm.precision == BIOT_FP32 ? "fp32" : "bf16", ctx->n_dof,
           ctx->wcap);
  const float* z = ctx->lp.Z;
  float* w = ctx->lp.Wv;
  auto time_v = [&](int v) -> double {
    const int save = ctx->spmm_var;
    ctx->spmm_var = v;
    const bool was = ctx->timing;
    ctx->timing = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, ctx->stream);
      launch_spmm_scaled<float>(ctx, z, w, 0, ctx->wcap);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = was;
    ctx->spmm_var = save;
    return best;
  };
  *ms_default = time_v(0);
  if (cache && cache->count(key)) {
    const int v = (*cache)[key];
    // the default shape (0) is always usable: it falls back to the scalar kernel when rows are not 16-byte aligned
    if (v >= 0 && v < kSpmmVariantCount && (v == 0 || spmm_variant_ok(ctx, v, z, w))) {
      ctx->spmm_var = v;
      *hit = 1;
      *ms_best = time_v(v);
      return BIOT_OK;
    }
  }
  int best = 0;
  double tbest = *ms_default;
  for (int v = 1; v < kSpmmVariantCount; ++v) {
    if (!spmm_variant_ok(ctx, v, z, w)) continue;
    const double t = time_v(v);
    if (t < tbest) {
      tbest = t;
      best = v;
    }
  }
  ctx->spmm_var = best;
  *ms_best = tbest;
  if (cache) (*cache)[key] = best;
  BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

}  // namespace biot
