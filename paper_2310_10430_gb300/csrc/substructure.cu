// Exact solves of the preconditioner blocks by one-level substructuring.
//
// P1 and P2 (Sec. 3.1, Eqs. p1, p2) need z_u = A^{-1} r_u and z_p = S^{-1} r_p with the
// elasticity block A (two DOFs per node) and the approximate Schur complement
// S = tau C + beta L (one DOF per node); the paper leaves the inner solvers open and this
// library solves them exactly. A plain band factorisation in natural node order has a
// half-band of about d (n + 2) and costs about 2 d (n + 2) flops per row and column per
// triangular solve. Here the mesh is cut by k - 1 vertical node lines (separators) into k
// strips of about (n + 2 - k) / k node columns. Ordering a strip's interior along its short
// side gives it a half-band of d (w + 2) - 1; the strips couple only through the separators.
// With I = all strip interiors and S = the separator DOFs:
//
//   z1 = A_II^{-1} r_I,   x_S = Ssep^{-1} (r_S - A_SI z1),   x_I = A_II^{-1} (r_I - A_IS x_S),
//   Ssep = A_SS - A_SI A_II^{-1} A_IS,
//
// which is exact (block Gaussian elimination). Ssep is block tridiagonal in separator order
// (strip t couples separators t - 1 and t), so it is stored and factored as one band of
// half-band 2 d (n + 1) - 1. The interior solves run all strips at once (grid.y = strip),
// many small CTAs per SM instead of one long band sweep per column pair. Setup forms
// A_II^{-1} A_IS strip-parallel with the same multi-right-hand-side band solves and
// subtracts A_SI (A_II^{-1} A_IS) from A_SS inside Ssep's band.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace biot {
namespace {

// natural block index o -> DOF (A: 2 v + f -> 3 v + f; S: v -> 3 v + 2)
template <int D> __device__ __forceinline__ int dof_of(int o) { return D == 2 ? 3 * (o >> 1) + (o & 1) : 3 * o + 2; }
// DOF c -> natural block index, or -1 if c is not in the block
template <int D> __device__ __forceinline__ int blk_of(int c) {
  const int f = c % 3;
  if (D == 2) return f == 2 ? -1 : 2 * (c / 3) + f;
  return f == 2 ? c / 3 : -1;
}
// the block's entries: A = AA_uu, S = -AA_pp
template <int D> __device__ __forceinline__ double sgn() { return D == 2 ? 1.0 : -1.0; }

struct SubArgs {
  int NI, NS, B, Ps, bI, bS;
  const int32_t* pos;
  const int32_t* oldI;
  const int32_t* oldS;
};
SubArgs args_of(const SubBlock* s) { return {s->NI, s->NS, s->B, s->Ps, s->bI, s->bS, s->pos, s->oldI, s->oldS}; }

// lower band of A_II (rows in the new interior order); padding rows get a unit diagonal
template <int D>
__global__ void k_sub_extract_I(SubArgs a, int nblk_old, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                double* __restrict__ LI, int32_t* __restrict__ err) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int ld = band_ld(a.bI);
  if (o < a.NI && a.oldI[o] < 0) LI[(size_t)o * ld + a.bI] = 1.0;  // o used as a new row index here
  if (o >= nblk_old) return;
  const int r = a.pos[o];
  if (r >= a.NI) return;
  const int dr = dof_of<D>(o);
  for (int32_t e = rowptr[dr]; e < rowptr[dr + 1]; ++e) {
    const int oc = blk_of<D>(col[e]);
    if (oc < 0) continue;
    const int cc = a.pos[oc];
    if (cc >= a.NI || cc > r) continue;
    if (r - cc > a.bI) {
      atomicExch(err, 1);
      continue;
    }
    LI[(size_t)r * ld + (a.bI - (r - cc))] = sgn<D>() * val[e];
  }
}

// Right-hand sides A_IS for strips t0 .. t0 + G - 1: Z[(row - t0 Ps)][col], column q of the
// strip's left separator (t - 1) at q, of its right separator (t) at B + q.
template <int D>
__global__ void k_sub_zrhs(SubArgs a, int t0, int G, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const double* __restrict__ val, double* __restrict__ Z,
                           int ldz, int32_t* __restrict__ err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.NS) return;
  const int m = s / a.B, q = s % a.B;
  const int dr = dof_of<D>(a.oldS[s]);
  for (int32_t e = rowptr[dr]; e < rowptr[dr + 1]; ++e) {
    const int oc = blk_of<D>(col[e]);
    if (oc < 0) continue;
    const int cc = a.pos[oc];
    if (cc >= a.NI) continue;
    const int t = cc / a.Ps;
    if (t < t0 || t >= t0 + G) continue;
    const int zc = (t == m) ? a.B + q : (t == m + 1 ? q : -1);
    if (zc < 0) {
      atomicExch(err, 2);
      continue;
    }
    Z[(size_t)(cc - t0 * a.Ps) * ldz + zc] = sgn<D>() * val[e];  // A symmetric: A_IS[i][s] = A[s][i]
  }
}

// Ssep's lower band starts as A_SS (separator-separator couplings lie on one line)
template <int D>
__global__ void k_sub_schur_init(SubArgs a, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ LS, int32_t* __restrict__ err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.NS) return;
  const int ld = band_ld(a.bS);
  const int dr = dof_of<D>(a.oldS[s]);
  for (int32_t e = rowptr[dr]; e < rowptr[dr + 1]; ++e) {
    const int oc = blk_of<D>(col[e]);
    if (oc < 0) continue;
    const int cc = a.pos[oc];
    if (cc < a.NI) continue;
    const int c2 = cc - a.NI;
    if (c2 > s) continue;
    if (s - c2 > a.bS) {
      atomicExch(err, 3);
      continue;
    }
    LS[(size_t)s * ld + (a.bS - (s - c2))] = sgn<D>() * val[e];
  }
}

// Ssep[s][c2] -= sum over interior i of strips t0 .. t0+G-1: A[s][i] (A_II^{-1} A_IS)[i][c2],
// one thread per band entry (s, q), c2 = s - bS + q, for the separator rows s0 <= s < s1 that
// border those strips (no other row has an interior neighbour in them).
template <int D>
__global__ void k_sub_schur_update(SubArgs a, int t0, int G, int s0, int s1, const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ col, const double* __restrict__ val,
                                   const double* __restrict__ Z, int ldz, double* __restrict__ LS) {
  const int ld = band_ld(a.bS);
  const long long tot = (long long)(s1 - s0) * (a.bS + 1);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int s = s0 + (int)(idx / (a.bS + 1)), q = (int)(idx % (a.bS + 1));
    const int c2 = s - a.bS + q;
    if (c2 < 0) continue;
    const int mc = c2 / a.B, qc = c2 % a.B;
    const int dr = dof_of<D>(a.oldS[s]);
    double acc = 0.0;
    for (int32_t e = rowptr[dr]; e < rowptr[dr + 1]; ++e) {
      const int oc = blk_of<D>(col[e]);
      if (oc < 0) continue;
      const int cc = a.pos[oc];
      if (cc >= a.NI) continue;
      const int t = cc / a.Ps;
      if (t < t0 || t >= t0 + G) continue;
      const int zc = (t == mc) ? a.B + qc : (t == mc + 1 ? qc : -1);
      if (zc < 0) continue;  // c2's separator does not border strip t
      acc += sgn<D>() * val[e] * Z[(size_t)(cc - t0 * a.Ps) * ldz + zc];
    }
    LS[(size_t)s * ld + q] -= acc;
  }
}

// ---- apply ----

// tI[r][c] = tI2[r][c] = rhs of interior row r, tS[s][c] = rhs of separator row s, for
// columns [c0, c0 + ncols). rhs: FROM_T ? tp[natural][c] : sgn * vin[dof][c] * sqrt|d_dof|.
template <int D, bool FROM_T, typename T>
__global__ void k_sub_gather(SubArgs a, const T* __restrict__ vin, const T* __restrict__ tp,
                             const double* __restrict__ dsq, T* __restrict__ tI, T* __restrict__ tI2,
                             T* __restrict__ tS, int ld, int c0, int ncols) {
  const int rows = a.NI + a.NS;
  const long long tot = (long long)rows * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    const int o = r < a.NI ? a.oldI[r] : a.oldS[r - a.NI];
    T v = T(0);
    if (o >= 0) {
      if (FROM_T) {
        v = tp[(size_t)o * ld + c];
      } else {
        const int dr = dof_of<D>(o);
        v = (T)sgn<D>() * vin[(size_t)dr * ld + c] * (T)dsq[dr];
      }
    }
    if (r < a.NI) {
      tI[(size_t)r * ld + c] = v;
      tI2[(size_t)r * ld + c] = v;
    } else {
      tS[(size_t)(r - a.NI) * ld + c] = v;
    }
  }
}

// tS[s][c] -= sum_i A[s][i] tI[i][c] over the interior neighbours i of separator row s
template <int D, typename T>
__global__ void k_sub_couple_S(SubArgs a, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const T* __restrict__ tI, T* __restrict__ tS, int ld,
                               int c0, int ncols) {
  const long long tot = (long long)a.NS * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    const int dr = dof_of<D>(a.oldS[s]);
    T acc = T(0);
    for (int32_t e = rowptr[dr]; e < rowptr[dr + 1]; ++e) {
      const int oc = blk_of<D>(col[e]);
      if (oc < 0) continue;
      const int cc = a.pos[oc];
      if (cc >= a.NI) continue;
      acc += (T)(sgn<D>() * val[e]) * tI[(size_t)cc * ld + c];
    }
    tS[(size_t)s * ld + c] -= acc;
  }
}

// tI2[r][c] -= sum_s A[r][s] tS[s][c] over the separator neighbours of the listed interior rows
template <int D, typename T>
__global__ void k_sub_couple_I(SubArgs a, const int32_t* __restrict__ adjI, int nadj,
                               const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const T* __restrict__ tS, T* __restrict__ tI2, int ld,
                               int c0, int ncols) {
  const long long tot = (long long)nadj * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = adjI[(int)(idx / ncols)], c = c0 + (int)(idx % ncols);
    const int dr = dof_of<D>(a.oldI[r]);
    T acc = T(0);
    for (int32_t e = rowptr[dr]; e < rowptr[dr + 1]; ++e) {
      const int oc = blk_of<D>(col[e]);
      if (oc < 0) continue;
      const int cc = a.pos[oc];
      if (cc < a.NI) continue;
      acc += (T)(sgn<D>() * val[e]) * tS[(size_t)(cc - a.NI) * ld + c];
    }
    tI2[(size_t)r * ld + c] -= acc;
  }
}

// z[dof][c] = solution (interior from tI2, separators from tS)
template <int D, typename T>
__global__ void k_sub_scatter(SubArgs a, const T* __restrict__ tI2, const T* __restrict__ tS, T* __restrict__ z,
                              int ld, int c0, int ncols) {
  const int rows = a.NI + a.NS;
  const long long tot = (long long)rows * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / ncols), c = c0 + (int)(idx % ncols);
    const int o = r < a.NI ? a.oldI[r] : a.oldS[r - a.NI];
    if (o < 0) continue;
    const T v = r < a.NI ? tI2[(size_t)r * ld + c] : tS[(size_t)(r - a.NI) * ld + c];
    z[(size_t)dof_of<D>(o) * ld + c] = v;
  }
}

// Offset of row r0's block in a variant's compact inverses (16 x 17 per 16 rows for the
// row-per-lane solve, nb x nb per nb rows otherwise).
size_t dnb_offset(int v, size_t r0) {
  return kBandVariants[v].tma == 3 ? r0 / 16 * 16 * 17 : r0 * (size_t)kBandVariants[v].nb;
}

int grid_for(long long work) { return (int)std::min<long long>(std::max<long long>((work + 255) / 256, 1), 152 * 16); }

// Strip widths and separator columns for k strips of the n + 1 node columns.
void layout(int n, int k, std::vector<int>& width, std::vector<int>& start, std::vector<int>& sep) {
  const int C = n + 1, ni = C - (k - 1);
  width.assign(k, ni / k);
  for (int t = 0; t < ni % k; ++t) ++width[t];
  start.assign(k, 0);
  sep.clear();
  int x = 0;
  for (int t = 0; t < k; ++t) {
    start[t] = x;
    x += width[t];
    if (t < k - 1) sep.push_back(x++);
  }
}

// First in-place variant that fits, in the given order of preference.
int pick_variant(bool fp64, int b, std::initializer_list<int> prefs) {
  for (int v : prefs)
    if (band_variant_inplace_ok(v, fp64, b)) return v;
  return -1;
}

template <int D>
biot_status setup_block(biot_ctx* ctx, int k, SubBlock*& out) {
  const int n = ctx->n, C = n + 1;
  std::vector<int> width, start, sep;
  layout(n, k, width, start, sep);
  SubBlock* sb = new (std::nothrow) SubBlock();
  if (!sb) return fail(ctx, BIOT_E_OOM, "substructure: host allocation");
  out = sb;
  sb->d = D;
  sb->k = k;
  sb->B = D * C;
  const int wmax = *std::max_element(width.begin(), width.end());
  sb->Ps = (D * wmax * C + 63) / 64 * 64;
  sb->NI = k * sb->Ps;
  sb->NS = (k - 1) * sb->B;
  sb->bI = D * (wmax + 2) - 1;
  sb->bS = 2 * sb->B - 1;
  const int nold = D * C * C;
  // orderings on the host
  std::vector<int> colstrip(C), collocal(C);
  for (int t = 0; t < k; ++t)
    for (int ii = 0; ii < width[t]; ++ii) {
      colstrip[start[t] + ii] = t;
      collocal[start[t] + ii] = ii;
    }
  for (int m = 0; m < k - 1; ++m) colstrip[sep[m]] = -1 - m;
  std::vector<int32_t> pos(nold), oldI(sb->NI, -1), oldS(sb->NS);
  std::vector<int32_t> adj;
  for (int j = 0; j < C; ++j)
    for (int i = 0; i < C; ++i)
      for (int f = 0; f < D; ++f) {
        const int o = D * (j * C + i) + f;
        const int cs = colstrip[i];
        if (cs >= 0) {
          const int r = cs * sb->Ps + D * (j * width[cs] + collocal[i]) + f;
          pos[o] = r;
          oldI[r] = o;
          // interior nodes next to a separator column couple to it
          if ((i > 0 && colstrip[i - 1] < 0) || (i + 1 < C && colstrip[i + 1] < 0)) adj.push_back(r);
        } else {
          const int s = (-1 - cs) * sb->B + D * j + f;
          pos[o] = sb->NI + s;
          oldS[s] = o;
        }
      }
  sb->nadj = (int)adj.size();
  cudaStream_t st = ctx->stream;
  const int ldI = band_ld(sb->bI), ldS = band_ld(sb->bS);
  const size_t nIrows = (size_t)sb->NI, nSrows = (size_t)(sb->NS + 63) / 64 * 64;
  const size_t szI = nIrows * ldI, szS = nSrows * ldS;
  const size_t dI = (size_t)div_up(sb->NI, kNB) * kNB * kNB, dS = (size_t)div_up(sb->NS, kNB) * kNB * kNB;
  BIOT_TRY(dalloc(ctx, (void**)&sb->pos, sizeof(int32_t) * nold));
  BIOT_TRY(dalloc(ctx, (void**)&sb->oldI, sizeof(int32_t) * sb->NI));
  BIOT_TRY(dalloc(ctx, (void**)&sb->oldS, sizeof(int32_t) * std::max(sb->NS, 1)));
  BIOT_TRY(dalloc(ctx, (void**)&sb->adjI, sizeof(int32_t) * std::max(sb->nadj, 1)));
  BIOT_TRY(dalloc(ctx, (void**)&sb->LI, sizeof(double) * szI));
  BIOT_TRY(dalloc(ctx, (void**)&sb->UI, sizeof(double) * szI));
  BIOT_TRY(dalloc(ctx, (void**)&sb->DI, sizeof(double) * dI));
  BIOT_TRY(dalloc(ctx, (void**)&sb->LS, sizeof(double) * szS));
  BIOT_TRY(dalloc(ctx, (void**)&sb->US, sizeof(double) * szS));
  BIOT_TRY(dalloc(ctx, (void**)&sb->DS, sizeof(double) * dS));
  BIOT_CU(ctx, cudaMemcpyAsync(sb->pos, pos.data(), sizeof(int32_t) * nold, cudaMemcpyHostToDevice, st));
  BIOT_CU(ctx, cudaMemcpyAsync(sb->oldI, oldI.data(), sizeof(int32_t) * sb->NI, cudaMemcpyHostToDevice, st));
  BIOT_CU(ctx, cudaMemcpyAsync(sb->oldS, oldS.data(), sizeof(int32_t) * sb->NS, cudaMemcpyHostToDevice, st));
  if (sb->nadj)
    BIOT_CU(ctx, cudaMemcpyAsync(sb->adjI, adj.data(), sizeof(int32_t) * sb->nadj, cudaMemcpyHostToDevice, st));
  BIOT_CU(ctx, cudaMemsetAsync(sb->LI, 0, sizeof(double) * szI, st));
  BIOT_CU(ctx, cudaMemsetAsync(sb->UI, 0, sizeof(double) * szI, st));
  BIOT_CU(ctx, cudaMemsetAsync(sb->LS, 0, sizeof(double) * szS, st));
  BIOT_CU(ctx, cudaMemsetAsync(sb->US, 0, sizeof(double) * szS, st));
  BIOT_CU(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), st));
  const SubArgs a = args_of(sb);
  // interior factor
  BIOT_LAUNCH(k_sub_extract_I<D>, div_up(std::max(nold, sb->NI), 256), 256, 0, st, a, nold, ctx->rowptr, ctx->col,
              ctx->val, sb->LI, ctx->status);
  {
    int32_t e = 0;
    BIOT_CU(ctx, cudaMemcpyAsync(&e, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BIOT_CU(ctx, cudaStreamSynchronize(st));
    if (e != 0) return fail(ctx, BIOT_E_CUDA, "substructure: interior entry outside the band (code %d)", e);
  }
  BIOT_TRY(band_factor(ctx, sb->NI, sb->bI, sb->LI, sb->UI, sb->DI));
  BIOT_CU(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), st));
  // variants: interior strips solved strip-parallel, separators as one band
  // defaults (biot_tune re-times them): the row-per-lane solve (7, one warp per CTA) only when
  // its one-warp CTAs cover every SM sub-partition, i.e. at least 4 x 152 of them (four columns
  // each, all strips); otherwise 128-thread split-row CTAs
  // Separators: the dense-block solve (separator.cu) by default; band substitutions (large
  // meshes: four-row blocks, the only staging that fits their half-band) stay available to
  // the tuner where one fits.
  const bool many = (long long)div_up(ctx->wcap, 4) * k >= 4 * 152;
  sb->varI[0] = many ? pick_variant(true, sb->bI, {7, 5, 1, 2, 3, 4}) : pick_variant(true, sb->bI, {5, 1, 2, 3, 4});
  sb->varS[0] = pick_variant(true, sb->bS, {5, 1, 2, 4, kWideVariant});
  sb->varI[1] = many ? pick_variant(false, sb->bI, {7, 5, 3, 1, 2, 4}) : pick_variant(false, sb->bI, {5, 3, 1, 2, 4});
  sb->varS[1] = pick_variant(false, sb->bS, {5, 3, 1, 2, 4, kWideVariant});
  const bool fp64 = ctx->prm.precision == BIOT_FP64;
  if (sb->varI[0] < 0 || sb->varI[1] < 0)
    return fail(ctx, BIOT_E_INVALID, "substructure: no band-solve variant fits the interiors' half-band %d", sb->bI);
  BIOT_TRY(dalloc(ctx, &sb->dnbI[0], sizeof(double) * ((size_t)sb->NI + 64) * 32));
  extract_dnb_variant<double>(ctx, sb->varI[0], sb->DI, sb->NI, (double*)sb->dnbI[0]);
  // Ssep = A_SS - A_SI A_II^{-1} A_IS, strips in groups that keep A_II^{-1} A_IS under 2 GB
  if (sb->NS > 0) {
    const int ldz = 2 * sb->B;
    const size_t per_strip = (size_t)sb->Ps * ldz * sizeof(double);
    const int G = (int)std::max<size_t>(1, std::min<size_t>((size_t)k, ((size_t)2 << 30) / per_strip));
    double* Z = nullptr;
    BIOT_TRY(dalloc(ctx, (void**)&Z, per_strip * G));
    BIOT_LAUNCH(k_sub_schur_init<D>, div_up(sb->NS, 256), 256, 0, st, a, ctx->rowptr, ctx->col, ctx->val, sb->LS,
                ctx->status);
    const size_t ldIsz = (size_t)ldI;
    for (int t0 = 0; t0 < k; t0 += G) {
      const int g = std::min(G, k - t0);
      BIOT_CU(ctx, cudaMemsetAsync(Z, 0, per_strip * g, st));
      BIOT_LAUNCH(k_sub_zrhs<D>, div_up(sb->NS, 256), 256, 0, st, a, t0, g, ctx->rowptr, ctx->col, ctx->val, Z, ldz,
                  ctx->status);
      const size_t r0 = (size_t)t0 * sb->Ps;
      const double* dnb = (const double*)sb->dnbI[0] + dnb_offset(sb->varI[0], r0);
      band_solve_inplace<double>(ctx, true, sb->varI[0], sb->Ps, g, sb->bI, sb->LI + r0 * ldIsz, dnb, Z, ldz, 0, ldz);
      band_solve_inplace<double>(ctx, false, sb->varI[0], sb->Ps, g, sb->bI, sb->UI + r0 * ldIsz, dnb, Z, ldz, 0, ldz);
      // strip t borders separators t - 1 and t
      const int s0 = std::max(t0 - 1, 0) * sb->B, s1 = std::min(t0 + g, k - 1) * sb->B;
      BIOT_LAUNCH(k_sub_schur_update<D>, grid_for((long long)(s1 - s0) * (sb->bS + 1)), 256, 0, st, a, t0, g, s0, s1,
                  ctx->rowptr, ctx->col, ctx->val, Z, ldz, sb->LS);
    }
    BIOT_CU(ctx, cudaGetLastError());
    BIOT_CU(ctx, cudaStreamSynchronize(st));
    int32_t e = 0;
    BIOT_CU(ctx, cudaMemcpy(&e, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (e != 0) return fail(ctx, BIOT_E_CUDA, "substructure: inconsistent ordering (code %d)", e);
    dfree(ctx, Z);
    BIOT_TRY(band_factor(ctx, sb->NS, sb->bS, sb->LS, sb->US, sb->DS));
    if (sb->varS[0] >= 0) {
      BIOT_TRY(dalloc(ctx, &sb->dnbS[0], sizeof(double) * ((size_t)sb->NS + 64) * 32));
      extract_dnb_variant<double>(ctx, sb->varS[0], sb->DS, sb->NS, (double*)sb->dnbS[0]);
    }
    BIOT_TRY(sep_dense_setup(ctx, sb));
  }
  if (ctx->prm.precision != BIOT_FP64) {
    // reduced-precision sweeps: the exact FP64 factors rounded to FP32
    BIOT_TRY(dalloc(ctx, (void**)&sb->LIf, sizeof(float) * szI));
    BIOT_TRY(dalloc(ctx, (void**)&sb->UIf, sizeof(float) * szI));
    BIOT_TRY(dalloc(ctx, (void**)&sb->DIf, sizeof(float) * dI));
    to_f32(ctx, sb->LI, sb->LIf, szI);
    to_f32(ctx, sb->UI, sb->UIf, szI);
    to_f32(ctx, sb->DI, sb->DIf, dI);
    BIOT_TRY(dalloc(ctx, &sb->dnbI[1], sizeof(float) * ((size_t)sb->NI + 64) * 32));
    extract_dnb_variant<float>(ctx, sb->varI[1], sb->DIf, sb->NI, (float*)sb->dnbI[1]);
    if (sb->NS > 0) {
      BIOT_TRY(dalloc(ctx, (void**)&sb->LSf, sizeof(float) * szS));
      BIOT_TRY(dalloc(ctx, (void**)&sb->USf, sizeof(float) * szS));
      BIOT_TRY(dalloc(ctx, (void**)&sb->DSf, sizeof(float) * dS));
      to_f32(ctx, sb->LS, sb->LSf, szS);
      to_f32(ctx, sb->US, sb->USf, szS);
      to_f32(ctx, sb->DS, sb->DSf, dS);
      if (sb->varS[1] >= 0) {
        BIOT_TRY(dalloc(ctx, &sb->dnbS[1], sizeof(float) * ((size_t)sb->NS + 64) * 32));
        extract_dnb_variant<float>(ctx, sb->varS[1], sb->DSf, sb->NS, (float*)sb->dnbS[1]);
      }
    }
  }
  if (sb->dense) {
    sb->varS[0] = sb->varS[1] = kDenseSep;
  } else if (sb->NS > 0 && ((fp64 && sb->varS[0] < 0) || sb->varS[1] < 0)) {
    return fail(ctx, BIOT_E_INVALID, "substructure: no separator solve fits half-band %d in %s", sb->bS,
                fp64 ? "FP64" : "FP32");
  }
  BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

template <typename T> struct SubFactors;
template <> struct SubFactors<double> {
  static const double* LI(const SubBlock* s) { return s->LI; }
  static const double* UI(const SubBlock* s) { return s->UI; }
  static const double* LS(const SubBlock* s) { return s->LS; }
  static const double* US(const SubBlock* s) { return s->US; }
  static constexpr int pi = 0;
};
template <> struct SubFactors<float> {
  static const float* LI(const SubBlock* s) { return s->LIf; }
  static const float* UI(const SubBlock* s) { return s->UIf; }
  static const float* LS(const SubBlock* s) { return s->LSf; }
  static const float* US(const SubBlock* s) { return s->USf; }
  static constexpr int pi = 1;
};

template <int D, typename T>
void apply_block(biot_ctx* ctx, SubBlock* sb, bool from_t, const T* vin, const T* tp, T* z, int c0, int ncols) {
  using F = SubFactors<T>;
  constexpr int pi = F::pi;
  const int ld = ctx->wcap;
  cudaStream_t st = ctx->stream;
  T* tI = (T*)sb->tI[pi];
  T* tI2 = (T*)sb->tI2[pi];
  T* tS = (T*)sb->tS[pi];
  const SubArgs a = args_of(sb);
  const long long rows = (long long)sb->NI + sb->NS;
  if (from_t)
    BIOT_LAUNCH((k_sub_gather<D, true, T>), grid_for(rows * ncols), 256, 0, st, a, vin, tp, ctx->dsq, tI, tI2, tS, ld,
                c0, ncols);
  else
    BIOT_LAUNCH((k_sub_gather<D, false, T>), grid_for(rows * ncols), 256, 0, st, a, vin, tp, ctx->dsq, tI, tI2, tS,
                ld, c0, ncols);
  const T* dnbI = (const T*)sb->dnbI[pi];
  const T* dnbS = (const T*)sb->dnbS[pi];
  // z1 = A_II^{-1} r_I
  band_solve_inplace<T>(ctx, true, sb->varI[pi], sb->Ps, sb->k, sb->bI, F::LI(sb), dnbI, tI, ld, c0, ncols);
  band_solve_inplace<T>(ctx, false, sb->varI[pi], sb->Ps, sb->k, sb->bI, F::UI(sb), dnbI, tI, ld, c0, ncols);
  if (sb->NS > 0) {
    // x_S = Ssep^{-1} (r_S - A_SI z1)
    BIOT_LAUNCH((k_sub_couple_S<D, T>), grid_for((long long)sb->NS * ncols), 256, 0, st, a, ctx->rowptr, ctx->col,
                ctx->val, tI, tS, ld, c0, ncols);
    if (sb->varS[pi] == kDenseSep) {
      sep_dense_solve<T>(ctx, sb, tS, (T*)sb->tZ[pi], ld, c0, ncols);
    } else {
      // Ssep is block tridiagonal with B x B blocks: its factor's band holds exact zeros to skip
      band_solve_inplace<T>(ctx, true, sb->varS[pi], sb->NS, 1, sb->bS, F::LS(sb), dnbS, tS, ld, c0, ncols, sb->B);
      band_solve_inplace<T>(ctx, false, sb->varS[pi], sb->NS, 1, sb->bS, F::US(sb), dnbS, tS, ld, c0, ncols, sb->B);
    }
    // x_I = A_II^{-1} (r_I - A_IS x_S)
    BIOT_LAUNCH((k_sub_couple_I<D, T>), grid_for((long long)sb->nadj * ncols), 256, 0, st, a, sb->adjI, sb->nadj,
                ctx->rowptr, ctx->col, ctx->val, tS, tI2, ld, c0, ncols);
    band_solve_inplace<T>(ctx, true, sb->varI[pi], sb->Ps, sb->k, sb->bI, F::LI(sb), dnbI, tI2, ld, c0, ncols);
    band_solve_inplace<T>(ctx, false, sb->varI[pi], sb->Ps, sb->k, sb->bI, F::UI(sb), dnbI, tI2, ld, c0, ncols);
  }
  BIOT_LAUNCH((k_sub_scatter<D, T>), grid_for(rows * ncols), 256, 0, st, a, sb->NS > 0 ? tI2 : tI, tS, z, ld, c0,
              ncols);
}

template <typename T>
biot_status ensure_workspace(biot_ctx* ctx, SubBlock* sb) {
  constexpr int pi = SubFactors<T>::pi;
  if (sb->tI[pi]) return BIOT_OK;
  const size_t w = (size_t)ctx->wcap;
  BIOT_TRY(dalloc(ctx, &sb->tI[pi], sizeof(T) * (size_t)sb->NI * w));
  BIOT_TRY(dalloc(ctx, &sb->tI2[pi], sizeof(T) * (size_t)sb->NI * w));
  BIOT_TRY(dalloc(ctx, &sb->tS[pi], sizeof(T) * ((size_t)std::max(sb->NS, 1)) * w));
  if (sb->dense) {
    BIOT_TRY(dalloc(ctx, &sb->tZ[pi], sizeof(T) * (size_t)sb->NS * w));
    BIOT_CU(ctx, cudaMemsetAsync(sb->tZ[pi], 0, sizeof(T) * (size_t)sb->NS * w, ctx->stream));
  }
  // padding rows and unused columns stay finite
  BIOT_CU(ctx, cudaMemsetAsync(sb->tI[pi], 0, sizeof(T) * (size_t)sb->NI * w, ctx->stream));
  BIOT_CU(ctx, cudaMemsetAsync(sb->tI2[pi], 0, sizeof(T) * (size_t)sb->NI * w, ctx->stream));
  BIOT_CU(ctx, cudaMemsetAsync(sb->tS[pi], 0, sizeof(T) * ((size_t)std::max(sb->NS, 1)) * w, ctx->stream));
  return BIOT_OK;
}

}  // namespace

// Strips for an n x n mesh when the caller leaves the choice open: about 18 node columns per
// strip in FP64 (k = 14 at n = 256, the fastest of k = 14 .. 28 with the dense separator
// solves) and about 10 in the reduced-precision sweeps (k = 26 at n = 256, fastest of 20 .. 40),
// none below n = 26 (FP64) or 13. Per column the interiors cost about d^2 (n + 1)^2 (w + 2)
// and the separators (k - 1) 1.5 d^2 (n + 1)^2, so the best k grows like sqrt(n + 1) rather
// than n: the count is capped at sqrt((n + 1) / c), c matched to the measured optima (1.31 in
// FP64 at n = 256; 0.38 in FP32, k = 52 at n = 1024 between the measured 40, 56 and 72).
int sub_auto_strips(int n, bool fp64) {
  const int lin = fp64 ? (n + 1 + 9) / 18 : (n + 1 + 6) / 10;
  const int cap = (int)std::lround(std::sqrt((n + 1) / (fp64 ? 1.31 : 0.38)));
  const int k = std::min(lin, cap);
  return k >= 2 ? k : 1;
}

int sub_strips(const biot_ctx* ctx) {
  const int k = ctx->sub_req == 0 ? sub_auto_strips(ctx->n, ctx->prm.precision == BIOT_FP64) : ctx->sub_req;
  return k >= 2 ? k : 1;
}

void sub_free(biot_ctx* ctx) {
  bool any = false;
  for (int w = 0; w < 2; ++w) any = any || ctx->sub[w];
  if (!any) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  for (int w = 0; w < 2; ++w) {
    SubBlock* sb = ctx->sub[w];
    if (!sb) continue;
    void* ptrs[] = {sb->pos, sb->oldI, sb->oldS, sb->adjI, sb->LI, sb->UI, sb->DI, sb->LS, sb->US, sb->DS,
                    sb->LIf, sb->UIf, sb->DIf, sb->LSf, sb->USf, sb->DSf, sb->dnbI[0], sb->dnbI[1],
                    sb->dnbS[0], sb->dnbS[1], sb->tI[0], sb->tI[1], sb->tI2[0], sb->tI2[1], sb->tS[0], sb->tS[1],
                    sb->Dinv, sb->Mk, sb->Pk, sb->Dinvf, sb->Mkf, sb->Pkf, sb->tZ[0], sb->tZ[1]};
    for (void* p : ptrs) dfree(ctx, p);
    delete sb;
    ctx->sub[w] = nullptr;
  }
}

biot_status sub_setup(biot_ctx* ctx) {
  sub_free(ctx);
  const int k = sub_strips(ctx);
  if (k < 2) return BIOT_OK;
  if (3 * k > ctx->n + 2) return fail(ctx, BIOT_E_INVALID, "substructure: %d strips leave fewer than 2 node columns per strip at n = %d", k, ctx->n);
  BIOT_TRY(setup_block<2>(ctx, k, ctx->sub[0]));
  BIOT_TRY(setup_block<1>(ctx, k, ctx->sub[1]));
  if (ctx->prm.precision == BIOT_FP64) {
    BIOT_TRY(ensure_workspace<double>(ctx, ctx->sub[0]));
    BIOT_TRY(ensure_workspace<double>(ctx, ctx->sub[1]));
  } else {
    BIOT_TRY(ensure_workspace<float>(ctx, ctx->sub[0]));
    BIOT_TRY(ensure_workspace<float>(ctx, ctx->sub[1]));
  }
  return BIOT_OK;
}

// which = 0: z_u = A^{-1} (d^{1/2} vin_u); which = 1: z_p = S^{-1} (-d^{1/2} vin_p) (P2), or
// S^{-1} tp when the caller passes vin = nullptr (P1: tp = B^T z_u - d^{1/2} vin_p).
template <typename T>
void sub_apply(biot_ctx* ctx, int which, const T* vin, T* z, int c0, int ncols) {
  if (which == 0) {
    apply_block<2, T>(ctx, ctx->sub[0], false, vin, nullptr, z, c0, ncols);
  } else {
    const T* tp = sizeof(T) == 8 ? (const T*)ctx->tp : (const T*)ctx->lp.tp;
    apply_block<1, T>(ctx, ctx->sub[1], vin == nullptr, vin, tp, z, c0, ncols);
  }
}
template void sub_apply<double>(biot_ctx*, int, const double*, double*, int, int);
template void sub_apply<float>(biot_ctx*, int, const float*, float*, int, int);

namespace {

// Forward + backward in-place solve pair of a substructured block's interiors (all strips)
// or separators, on its workspace at full window width; best of two timed repetitions.
template <typename T>
float time_sub_pair(biot_ctx* ctx, SubBlock* sb, bool interior, int v) {
  using F = SubFactors<T>;
  constexpr int pi = F::pi;
  const int N = interior ? sb->Ps : sb->NS, nst = interior ? sb->k : 1, b = interior ? sb->bI : sb->bS;
  const T* L = interior ? F::LI(sb) : F::LS(sb);
  const T* U = interior ? F::UI(sb) : F::US(sb);
  const T* dnb = (const T*)(interior ? sb->dnbI[pi] : sb->dnbS[pi]);
  T* buf = (T*)(interior ? sb->tI[pi] : sb->tS[pi]);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, ctx->stream);
    const int blk = interior ? 0 : sb->B;
    if (v == kDenseSep) {
      sep_dense_solve<T>(ctx, sb, buf, (T*)sb->tZ[pi], ctx->wcap, 0, ctx->wcap);
    } else {
      band_solve_inplace<T>(ctx, true, v, N, nst, b, L, dnb, buf, ctx->wcap, 0, ctx->wcap, blk);
      band_solve_inplace<T>(ctx, false, v, N, nst, b, U, dnb, buf, ctx->wcap, 0, ctx->wcap, blk);
    }
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

template <typename T>
void set_dnb(biot_ctx* ctx, SubBlock* sb, bool interior, int v) {
  constexpr int pi = SubFactors<T>::pi;
  if (v == kDenseSep || (!interior && !sb->dnbS[pi])) return;
  const T* D = (const T*)(interior ? (pi ? (const void*)sb->DIf : (const void*)sb->DI)
                                   : (pi ? (const void*)sb->DSf : (const void*)sb->DS));
  extract_dnb_variant<T>(ctx, v, D, interior ? sb->NI : sb->NS, (T*)(interior ? sb->dnbI[pi] : sb->dnbS[pi]));
}

template <typename T>
float tune_part(biot_ctx* ctx, SubBlock* sb, bool interior, std::map<std::string, int>* cache, int* hits) {
  constexpr int pi = SubFactors<T>::pi;
  const bool fp64 = pi == 0;
  int& var = interior ? sb->varI[pi] : sb->varS[pi];
  const int b = interior ? sb->bI : sb->bS;
  char key[96];
  snprintf(key, sizeof(key), "sub:%s:N%d:b%d:w%d", fp64 ? "fp64" : "fp32", interior ? sb->NI : sb->NS, b, ctx->wcap);
  auto usable = [&](int v) {
    if (v == kDenseSep) return !interior && sb->dense;
    return band_variant_inplace_ok(v, fp64, b) && (interior || sb->dnbS[pi] != nullptr);
  };
  if (cache && cache->count(key) && usable((*cache)[key])) {
    var = (*cache)[key];
    set_dnb<T>(ctx, sb, interior, var);
    ++*hits;
    return time_sub_pair<T>(ctx, sb, interior, var);
  }
  float tbest = time_sub_pair<T>(ctx, sb, interior, var);
  int best = var;
  std::vector<int> cands;
  for (int v = 1; v < kBandVariantCount; ++v) cands.push_back(v);
  cands.push_back(kDenseSep);
  for (int v : cands) {
    if (v == var || !usable(v)) continue;
    set_dnb<T>(ctx, sb, interior, v);
    const float t = time_sub_pair<T>(ctx, sb, interior, v);
    if (t < tbest) {
      tbest = t;
      best = v;
    }
  }
  var = best;
  set_dnb<T>(ctx, sb, interior, best);
  if (cache) (*cache)[key] = best;
  return tbest;
}

}  // namespace

// Times every fitting TMA variant for the strip interiors and for the separators of A and
// S and keeps the fastest; ms[0], ms[1]: the chosen interior + separator pair times of A, S,
// ms_sep[0], ms_sep[1]: their separator parts.
biot_status sub_tune(biot_ctx* ctx, double* ms, double* ms_sep, std::map<std::string, int>* cache, int* hits) {
  const bool fp64 = ctx->prm.precision == BIOT_FP64;
  *hits = 0;
  for (int w = 0; w < 2; ++w) {
    SubBlock* sb = ctx->sub[w];
    ms[w] = ms_sep[w] = 0.0;
    if (!sb) continue;
    ms[w] += fp64 ? tune_part<double>(ctx, sb, true, cache, hits) : tune_part<float>(ctx, sb, true, cache, hits);
    if (sb->NS > 0)
      ms_sep[w] = fp64 ? tune_part<double>(ctx, sb, false, cache, hits) : tune_part<float>(ctx, sb, false, cache, hits);
    else
      ++*hits;  // no separators: nothing to choose
    ms[w] += ms_sep[w];
  }
  BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

}  // namespace biot
