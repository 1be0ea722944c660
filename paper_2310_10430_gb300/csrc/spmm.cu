// Multi-right-hand-side sparse products of the sweep (FP64).
//
// The residual of every active time step (Alg. 3: b^{n,m} = A' X^{n-1,m} + f^n,
// r = b - AA X^{n,m-1}) is formed in one pass over the matrix: a warp owns one
// mesh node (three CSR rows: u_x, u_y, p) and its lanes own consecutive time
// steps. The state X is stored [DOF][time] (time fastest), so a warp's loads of
// X[dof][lo-1 .. hi] are contiguous. Each 3x3 node block of AA is read once per
// node and applied to all active steps; A' shares B^T with AA and adds its own
// pressure-pressure entry, applied to X at step n-1.
#include "common.cuh"

namespace biot {

namespace {

constexpr int kWarps = 8;

// Reduce one double per (warp, lane) over the block's warps in warp order and
// store it at dst[lane] (called by all threads; dst may be null for lanes >= count).
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

__global__ void __launch_bounds__(kWarps * 32)
k_residual(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
           const int32_t* __restrict__ rowptr, const double* __restrict__ val, const double* __restrict__ apval,
           const double* __restrict__ dsc, const double* __restrict__ X, const double* __restrict__ F, int ldx, int lo,
           int ncols, double* __restrict__ out, int ldo, double* __restrict__ part, int ldp) {
  __shared__ double sm[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nn + gridDim.x - 1) / gridDim.x;
  const int vb = blockIdx.x * per, ve = min(nn, vb + per);
  for (int cb = 0; cb < ncols; cb += 32) {
    const int c = cb + lane;
    const bool cv = c < ncols;
    const int tn = lo + (cv ? c : 0);  // time step of this lane
    double rr = 0.0, bb = 0.0;
    for (int v = vb + warp; v < ve; v += kWarps) {
      const int32_t np = nodeptr[v];
      const int deg = nodeptr[v + 1] - np;
      const int32_t r0 = rowptr[3 * v], r1 = r0 + 3 * deg, r2 = r1 + 3 * deg;
      const double f0 = F[(size_t)(3 * v) * ldx + tn];
      const double f1 = F[(size_t)(3 * v + 1) * ldx + tn];
      const double f2 = F[(size_t)(3 * v + 2) * ldx + tn];
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, ap = 0.0;
      for (int k = 0; k < deg; ++k) {
        const int m = nbr[np + k];
        const double* xm = X + (size_t)(3 * m) * ldx + tn;
        const double x0 = xm[0], x1 = xm[ldx], x2 = xm[2 * ldx];
        const double y0 = xm[-1], y1 = xm[ldx - 1], y2 = xm[2 * ldx - 1];
        const double* e0 = val + r0 + 3 * k;
        const double* e1 = val + r1 + 3 * k;
        const double* e2 = val + r2 + 3 * k;
        a0 += e0[0] * x0 + e0[1] * x1 + e0[2] * x2;
        a1 += e1[0] * x0 + e1[1] * x1 + e1[2] * x2;
        a2 += e2[0] * x0 + e2[1] * x1 + e2[2] * x2;
        ap += e2[0] * y0 + e2[1] * y1 + apval[np + k] * y2;
      }
      const double d0 = dsc[3 * v], d1 = dsc[3 * v + 1], d2 = dsc[3 * v + 2];
      const double b2 = f2 + ap;
      const double q0 = d0 * (f0 - a0), q1 = d1 * (f1 - a1), q2 = d2 * (b2 - a2);
      if (cv) {
        out[(size_t)(3 * v) * ldo + c] = q0;
        out[(size_t)(3 * v + 1) * ldo + c] = q1;
        out[(size_t)(3 * v + 2) * ldo + c] = q2;
        rr += q0 * q0 + q1 * q1 + q2 * q2;
        const double p0 = d0 * f0, p1 = d1 * f1, p2 = d2 * b2;
        bb += p0 * p0 + p1 * p1 + p2 * p2;
      }
    }
    block_sum_to(sm, rr, part + (size_t)(0 * gridDim.x + blockIdx.x) * ldp + cb, min(32, ncols - cb));
    block_sum_to(sm, bb, part + (size_t)(1 * gridDim.x + blockIdx.x) * ldp + cb, min(32, ncols - cb));
  }
}

// w[:, c] = d .* (AA z[:, c]) for c in [c0, c0 + ncols); partial |w|^2 in slot 0.
__global__ void __launch_bounds__(kWarps * 32)
k_spmm_scaled(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
              const int32_t* __restrict__ rowptr, const double* __restrict__ val, const double* __restrict__ dsc,
              const double* __restrict__ z, double* __restrict__ w, int ld, int c0, int ncols,
              double* __restrict__ part) {
  __shared__ double sm[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nn + gridDim.x - 1) / gridDim.x;
  const int vb = blockIdx.x * per, ve = min(nn, vb + per);
  for (int cb = 0; cb < ncols; cb += 32) {
    const int c = c0 + cb + lane;
    const bool cv = cb + lane < ncols;
    const int cc = cv ? c : c0;
    double ww = 0.0;
    for (int v = vb + warp; v < ve; v += kWarps) {
      const int32_t np = nodeptr[v];
      const int deg = nodeptr[v + 1] - np;
      const int32_t r0 = rowptr[3 * v], r1 = r0 + 3 * deg, r2 = r1 + 3 * deg;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (int k = 0; k < deg; ++k) {
        const int m = nbr[np + k];
        const double* zm = z + (size_t)(3 * m) * ld + cc;
        const double x0 = zm[0], x1 = zm[ld], x2 = zm[2 * ld];
        const double* e0 = val + r0 + 3 * k;
        const double* e1 = val + r1 + 3 * k;
        const double* e2 = val + r2 + 3 * k;
        a0 += e0[0] * x0 + e0[1] * x1 + e0[2] * x2;
        a1 += e1[0] * x0 + e1[1] * x1 + e1[2] * x2;
        a2 += e2[0] * x0 + e2[1] * x1 + e2[2] * x2;
      }
      const double q0 = dsc[3 * v] * a0, q1 = dsc[3 * v + 1] * a1, q2 = dsc[3 * v + 2] * a2;
      if (cv) {
        w[(size_t)(3 * v) * ld + c] = q0;
        w[(size_t)(3 * v + 1) * ld + c] = q1;
        w[(size_t)(3 * v + 2) * ld + c] = q2;
        ww += q0 * q0 + q1 * q1 + q2 * q2;
      }
    }
    block_sum_to(sm, ww, part + (size_t)blockIdx.x * ld + c0 + cb, min(32, ncols - cb));
  }
}

// P1 coupling: tp[v][c] = (B^T z_u)[v][c] - vin[3v+2][c] / d[3v+2].
__global__ void k_coupling(int nn, const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
                           const int32_t* __restrict__ rowptr, const double* __restrict__ val,
                           const double* __restrict__ dsc, const double* __restrict__ z,
                           const double* __restrict__ vin, double* __restrict__ tp, int ld, int c0, int ncols) {
  const int c = c0 + (int)(threadIdx.x % 32) + 32 * (int)(blockIdx.y);
  const int v = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (v >= nn || c >= c0 + ncols) return;
  const int32_t np = nodeptr[v];
  const int deg = nodeptr[v + 1] - np;
  const int32_t r2 = rowptr[3 * v] + 6 * deg;
  double s = 0.0;
  for (int k = 0; k < deg; ++k) {
    const int m = nbr[np + k];
    s += val[r2 + 3 * k] * z[(size_t)(3 * m) * ld + c] + val[r2 + 3 * k + 1] * z[(size_t)(3 * m + 1) * ld + c];
  }
  tp[(size_t)v * ld + c] = s - vin[(size_t)(3 * v + 2) * ld + c] / dsc[3 * v + 2];
}

}  // namespace

void launch_residual_raw(int n_nodes, const int32_t* nodeptr, const int32_t* nbr, const int32_t* rowptr,
                         const double* val, const double* apval, const double* dsc, const double* X,
                         const double* F, int ldx, int lo, int ncols, double* out, int ldo, double* part, int ldp,
                         cudaStream_t stream) {
  BIOT_LAUNCH(k_residual, kRedBlocks, kWarps * 32, 0, stream, n_nodes, nodeptr, nbr, rowptr, val, apval, dsc, X, F,
              ldx, lo, ncols, out, ldo, part, ldp);
}

void launch_residual(biot_ctx* ctx, int lo, int ncols, double* out, int ldo) {
  KTimer tm(ctx, BIOT_KC_RESIDUAL);
  BIOT_LAUNCH(k_residual, kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr, ctx->nbr, ctx->rowptr,
              ctx->val, ctx->apval, ctx->dsc, ctx->X, ctx->F, ctx->ldx, lo, ncols, out, ldo, ctx->part, ctx->wcap);
}

void launch_spmm_scaled(biot_ctx* ctx, const double* z, double* w, int c0, int ncols) {
  KTimer tm(ctx, BIOT_KC_SPMM);
  BIOT_LAUNCH(k_spmm_scaled, kRedBlocks, kWarps * 32, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr, ctx->nbr,
              ctx->rowptr, ctx->val, ctx->dsc, z, w, ctx->wcap, c0, ncols, ctx->part);
}

void launch_coupling(biot_ctx* ctx, const double* z, const double* vin, double* tp, int c0, int ncols) {
  dim3 grid(div_up(ctx->n_nodes, 8), div_up(ncols, 32));
  BIOT_LAUNCH(k_coupling, grid, 256, 0, ctx->stream, ctx->n_nodes, ctx->nodeptr, ctx->nbr, ctx->rowptr, ctx->val,
              ctx->dsc, z, vin, tp, ctx->wcap, c0, ncols);
}

}  // namespace biot
