// Internal declarations shared by the CUDA translation units of the Biot PinT
// library. Nothing here is part of the public ABI (include/biot_pint.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/biot_pint.h"

namespace biot {

struct Gmg;  // multigrid hierarchy of the block solves (gmg.cu)

// Kernel launches issued by the library (reported by biot_launch_count).
extern std::atomic<int64_t> g_launches;

// Launch helper: counts the launch and records launch-configuration errors.
#define BIOT_LAUNCH(kernel, grid, block, smem, stream, ...)              \
  do {                                                                   \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);          \
    ::biot::g_launches.fetch_add(1, std::memory_order_relaxed);          \
  } while (0)

// Fixed reduction grid: partial sums per block are reduced in a second pass in
// block order, so every norm and dot product is deterministic.
constexpr int kRedBlocks = 304;         // 2 x 152 SMs
constexpr int kDotBlocks = 456;         // 3 x 152 SMs: the FP32 Gram-Schmidt dot products' grid (three CTAs per SM)
constexpr int kPartBlocks = kDotBlocks > kRedBlocks ? kDotBlocks : kRedBlocks;
constexpr int kMaxIter = 32;            // n_iter upper bound
constexpr double kBreakdownRtol = 1e-14;  // lucky-breakdown test h_{j+1,j} <= rtol |A z_j|

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Buffers of the reduced-precision sweep (FP32 Krylov vectors; BF16 or FP32 matrix
// values): every sweep forms the true residual in FP64, runs the FGMRES cycle in FP32
// on the correction and adds it to the FP64 state (iterative refinement per sweep).
struct LowPrec {
  float* V = nullptr;            // (n_iter + 1) x [n_dof][wcap]
  float* Z = nullptr;            // n_iter x [n_dof][wcap]
  float* Wv = nullptr;           // [n_dof][wcap]
  float* tu = nullptr;           // [2 n_nodes][wcap]
  float* tp = nullptr;           // [n_nodes][wcap]
  float* val = nullptr;          // AA values (CSR order)
  float* apval = nullptr;        // A' pressure-pressure values (node-pair order)
  __nv_bfloat16* val_bf16 = nullptr;
  __nv_bfloat16* apval_bf16 = nullptr;
  float* Lu = nullptr;           // band factors rounded from the FP64 factorisation
  float* Uu = nullptr;
  float* Du = nullptr;
  float* Lp = nullptr;
  float* Up = nullptr;
  float* Dp = nullptr;
  float* tile[2][2] = {};        // [u, p][forward, backward]: skewed block tiles of the band solve
  int tile_ok[2] = {0, 0};       // tiles of [u, p] built from the current factors
  float* bdnb[2] = {nullptr, nullptr};  // [u, p] compact block inverses for the batched solve
  int bdnb_ok = 0;
};

// One instance of a batch, as the batched kernels see it (device-resident table).
// Window: residual columns [0, nres) for steps lo .. lo + nres - 1; FGMRES on
// columns [c0, c0 + nf).
struct InstDev {
  int n_nodes, n_dof, ldx, wcap, n_t, band_u, band_p;
  int lo, nres, c0, nf, active;
  const int32_t* nodeptr;
  const int32_t* nbr;
  const int32_t* rowptr;
  const double* dsc;
  const double* val64;
  const double* apval64;
  const double* X64;
  const double* F64;
  double* X64w;
  const float* val;
  const float* apval;
  const __nv_bfloat16* valbf;
  const __nv_bfloat16* apvalbf;
  float* V;
  float* Z;
  float* Wv;
  float* tu;
  float* tp;
  const float* Lu;
  const float* Uu;
  const float* Du;
  const float* Lp;
  const float* Up;
  const float* Dp;
  const double* dsq;
  const float* dnbu;    // compact 32 x 32 block inverses of A's and S's FP32 factors
  const float* dnbp;
  int32_t* status;      // the instance context's device error flag
  double* part;
  double* colscal;
  double* H;
  double* hvec;
  int32_t* kcol;
};

}  // namespace biot

// Rows per block of the band solves' diagonal-block inverses (and of the legacy solve).
constexpr int kNB = 64;
// Leading dimension of the band rows: b + 1 entries padded to a multiple of 4, so every
// row starts on a 16-byte boundary (vector loads, whole-block bulk copies).
__host__ __device__ constexpr int band_ld(int b) { return (b + 1 + 3) & ~3; }

// Exact solve of one preconditioner block (A: d = 2 DOFs per node, S: d = 1) by one-level
// substructuring: k strips of node columns separated by k - 1 separator node columns
// (substructure.cu). New order: strip interiors (strip t at rows t Ps .., x fastest within
// the strip, padded to Ps rows with identity rows), then separators (line by line, along y).
struct SubBlock {
  int d = 0, k = 0;                 // DOFs per node, strips
  int B = 0;                        // DOFs per separator line: d (n + 1)
  int Ps = 0, NI = 0, NS = 0;       // rows per strip (multiple of 64), k Ps, (k - 1) B
  int bI = 0, bS = 0;               // half-bands of the interior factor and of the separator Schur complement
  int nadj = 0;                     // interior rows coupled to a separator
  int32_t* pos = nullptr;           // [d (n+1)^2] natural block index -> new index (NI + s for separators)
  int32_t* oldI = nullptr;          // [NI] new interior row -> natural block index (-1: padding)
  int32_t* oldS = nullptr;          // [NS]
  int32_t* adjI = nullptr;          // [nadj] interior rows coupled to a separator
  double *LI = nullptr, *UI = nullptr, *DI = nullptr, *LS = nullptr, *US = nullptr, *DS = nullptr;
  float *LIf = nullptr, *UIf = nullptr, *DIf = nullptr, *LSf = nullptr, *USf = nullptr, *DSf = nullptr;
  void* dnbI[2] = {nullptr, nullptr};  // compact block inverses for the chosen variants [FP64, FP32]
  void* dnbS[2] = {nullptr, nullptr};
  int varI[2] = {0, 0}, varS[2] = {0, 0};  // TMA band-solve variants [FP64, FP32]
  void* tI[2] = {nullptr, nullptr};       // workspaces [NI][wcap], [NI][wcap], [NS][wcap] per precision
  void* tI2[2] = {nullptr, nullptr};
  void* tS[2] = {nullptr, nullptr};
  // dense-block separator solves (separator.cu): D_K^{-1}, M_K, P_K as Bp x Bp blocks
  bool dense = false;
  int Bp = 0;                       // B rounded up to a multiple of 64
  double *Dinv = nullptr, *Mk = nullptr, *Pk = nullptr;
  float *Dinvf = nullptr, *Mkf = nullptr, *Pkf = nullptr;
  void* tZ[2] = {nullptr, nullptr};       // [NS][wcap] forward results per precision
};

struct biot_ctx {
  // mesh
  int n = 0;
  double Lx = 1.0, Ly = 1.0;
  cudaStream_t stream = nullptr;
  // P2's two block solves run concurrently: A's on `side` (highest priority), S's on `stream`
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // substructured block solves: requested strip count (0 automatic, 1 off, >= 2 forced)
  // and the set-up blocks [A, S] (null: plain band solves)
  int sub_req = 0;
  SubBlock* sub[2] = {nullptr, nullptr};
  int n_nodes = 0, n_dof = 0, n_pairs = 0;
  int64_t nnz = 0;
  // pattern (device)
  int32_t* nodeptr = nullptr;   // [n_nodes + 1]
  int32_t* nbr = nullptr;       // [n_pairs] sorted neighbour lists (self included)
  int32_t* rowptr = nullptr;    // [n_dof + 1]
  int32_t* col = nullptr;       // [nnz]
  // values (device, FP64)
  double* val = nullptr;        // AA after Dirichlet elimination, CSR order
  double* apval = nullptr;      // A'_pp after elimination, node-pair order
  double* dsc = nullptr;        // d = |diag AA|^{-1/2}
  double* dsq = nullptr;        // |diag AA|^{1/2}: multiplies instead of dividing by dsc
  uint8_t* dmask = nullptr;     // 1 on Dirichlet DOFs
  double* kappa = nullptr;      // [2 n^2]
  // time data
  int n_t = 0;
  int ldx = 0;                  // leading dimension of X and F (>= n_t + 1)
  double* X = nullptr;          // [n_dof][ldx], column n = step n
  double* F = nullptr;          // [n_dof][ldx], column 0 zero
  // Krylov work buffers, [n_dof][wcap] each
  int wcap = 0;
  int n_iter = 0;
  double* V = nullptr;          // (n_iter + 1) vectors
  double* Z = nullptr;          // n_iter vectors
  double* Wv = nullptr;         // Arnoldi candidate w
  double* part = nullptr;       // [kPartBlocks][(kMaxIter + 2)][wcap] partial sums
  double* colscal = nullptr;    // per-column scalars: see krylov.cu (layout kColScalars x wcap)
  double* H = nullptr;          // [wcap][(kMaxIter + 1) * kMaxIter]
  double* hvec = nullptr;       // [kMaxIter + 1][wcap] reduced dots of the current step
  int32_t* kcol = nullptr;      // [wcap] Arnoldi steps taken per column
  // band preconditioner
  int band_u = 0, band_p = 0;
  int precond = 0;
  bool plain_band = true;       // natural-order band factors built (false: large substructured meshes)
  double* Lu = nullptr;         // A = L L^T, lower band rows [2 n_nodes][band_u + 1]
  double* Uu = nullptr;         // L^T band rows [2 n_nodes][band_u + 1]
  double* Lp = nullptr;         // S = L L^T, [n_nodes][band_p + 1]
  double* Up = nullptr;
  double* Du = nullptr;         // inverses of the 64 x 64 diagonal blocks of L (A)
  double* Dp = nullptr;         // same for S
  double* tu = nullptr;         // [2 n_nodes][wcap] forward-solve scratch (u)
  double* tp = nullptr;         // [n_nodes][wcap] coupling / forward scratch (p)
  int32_t* status = nullptr;    // device status word (factorisation pivots)
  biot::LowPrec lp;             // reduced-precision sweep buffers (BIOT_FP32 / BIOT_BF16VAL_FP32ACC)
  int band_var_u[2] = {0, 0};   // band-solve variant for A, [FP64, FP32] (kBandVariants index)
  int band_var_p[2] = {0, 0};   // same for S
  int spmm_var = 0;             // tuned shape of the FP32 / BF16-value SpMM (spmm.cu)
  void* dnb_u[2] = {nullptr, nullptr};  // compact NB x NB diagonal-block inverses of A, [FP64, FP32]
  void* dnb_p[2] = {nullptr, nullptr};  // same for S
  int dnb_nb_u[2] = {0, 0};     // NB they were built for (0: none)
  int dnb_nb_p[2] = {0, 0};
  // inner solver of the block solves: exact (band / substructured) or multigrid V-cycles
  int inner = BIOT_INNER_EXACT;
  int gmg_levels_req = 0, gmg_cycles = 1, gmg_smooth = 2;
  biot::Gmg* gmg = nullptr;
  double beta_force = -1.0;     // >= 0: stabilisation factor to use instead of the mesh's own
  // params
  biot_params prm{};
  double beta = 0.0;
  bool assembled = false;
  // per-class event timing (biot_timing_enable / biot_timing_read)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<size_t, size_t>> ev_marks[BIOT_KC_COUNT];
  // bookkeeping
  int64_t device_bytes = 0;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;
  std::string err;
};

namespace biot {

// Brackets the launches issued in its scope with CUDA events when timing is on.
struct KTimer {
  biot_ctx* ctx;
  int kc;
  size_t a = 0;
  KTimer(biot_ctx* c, int k);
  ~KTimer();
};

// Error plumbing: every failing call stores a message in ctx->err.
biot_status fail(biot_ctx* ctx, biot_status st, const char* fmt, ...);
biot_status cuda_check(biot_ctx* ctx, cudaError_t e, const char* what);
biot_status dalloc(biot_ctx* ctx, void** p, size_t bytes);
void dfree(biot_ctx* ctx, void* p);  // one dalloc'ed block (the stream must not still use it)
void dfree_all(biot_ctx* ctx);

#define BIOT_CU(ctx, call)                                                   \
  do {                                                                       \
    biot_status _st = ::biot::cuda_check((ctx), (call), #call);              \
    if (_st != BIOT_OK) return _st;                                          \
  } while (0)
#define BIOT_TRY(call)                                                       \
  do {                                                                       \
    biot_status _st = (call);                                                \
    if (_st != BIOT_OK) return _st;                                          \
  } while (0)

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---- band.cu: building blocks shared with the substructured solves ----
biot_status band_factor(biot_ctx* ctx, int N, int b, double* L, double* U, double* D);
template <typename T>
void band_solve_inplace(biot_ctx* ctx, bool fwd, int variant, int N, int nstrips, int b, const T* band,
                        const T* Dnb, T* buf, int ld, int c0, int ncols, int blk = 0);  // blk: see the body
template <typename T> void extract_dnb_raw(biot_ctx* ctx, const T* D64, int N, int nb, T* out);
template <typename T> void extract_dnb_variant(biot_ctx* ctx, int variant, const T* D64, int N, T* out);
void to_f32(biot_ctx* ctx, const double* in, float* out, size_t n);

// ---- substructure.cu ----
int sub_auto_strips(int n, bool fp64);
int sub_strips(const biot_ctx* ctx);  // strips sub_setup will use (1: natural-order band solves)
biot_status sub_setup(biot_ctx* ctx);
void sub_free(biot_ctx* ctx);
template <typename T> void sub_apply(biot_ctx* ctx, int which, const T* vin, T* z, int c0, int ncols);
// ---- separator.cu ----
biot_status sep_dense_setup(biot_ctx* ctx, SubBlock* sb);  // needs sb->LS factored
template <typename T> void sep_dense_solve(biot_ctx* ctx, SubBlock* sb, T* tS, T* tZ, int ld, int c0, int ncols);
biot_status sub_tune(biot_ctx* ctx, double* ms, double* ms_sep, std::map<std::string, int>* cache, int* hits);

// ---- gmg.cu ----
biot_status gmg_setup(biot_ctx* ctx);
void gmg_free(biot_ctx* ctx);
int gmg_levels_for(int n, int req);
template <typename T> void gmg_apply(biot_ctx* ctx, const T* vin, T* z, int c0, int ncols);
void gmg_info(const biot_ctx* ctx, int* levels, double* lam_u, double* lam_p);

// ---- assembly.cu ----
biot_status build_pattern(biot_ctx* ctx);
biot_status assemble_system(biot_ctx* ctx);

// ---- spmm.cu ----
// FP64 window residual: out[:, c] = d .* (F[:, lo+c] + A' X[:, lo+c-1] - AA X[:, lo+c]), c < ncols;
// partials of |d r|^2 and |d b|^2 per column into part (slots 0 and 1).
void launch_residual(biot_ctx* ctx, int lo, int ncols, double* out, int ldo);
// The same kernel on caller-given buffers; partials to part[2][kRedBlocks][ldp].
void launch_residual_raw(int n_nodes, const int32_t* nodeptr, const int32_t* nbr, const int32_t* rowptr,
                         const double* val, const double* apval, const double* dsc, const double* X,
                         const double* F, int ldx, int lo, int ncols, double* out, int ldo, double* part, int ldp,
                         cudaStream_t stream);
// FP64 true residual of the window written equilibrated into the FP32 lp.V.
void launch_residual_lp(biot_ctx* ctx, int lo, int ncols);
// w = d .* (AA z) for columns [c0, c0 + ncols); partial |w|^2 into slot 0.
template <typename T> void launch_spmm_scaled(biot_ctx* ctx, const T* z, T* w, int c0, int ncols);
// Norm partials per column the SpMM writes (its grid), and the SpMM shape tuner.
int spmm_blocks(const biot_ctx* ctx);
biot_status spmm_tune(biot_ctx* ctx, std::map<std::string, int>* cache, int* hit, double* ms_best,
                      double* ms_default);
// t_p[v][c] = sum_m B^T[v][m] z_u[m][c] - v_p[v][c]/d (P1 coupling).
template <typename T> void launch_coupling(biot_ctx* ctx, const T* z, const T* vin, T* tp, int c0, int ncols);

// ---- band.cu ----
struct BandVariant {
  int tma;      // 1: band rows staged in shared memory by bulk copies; 2: skewed block tiles (FP32);
                // 3: row per lane, in-place strip solves only
  int nb;       // rows per block
  int threads;  // CTA size
};
constexpr int kBandVariantCount = 11;
// Four-row blocks: the only TMA variant whose two band stages fit beside the ring at the
// separators' half-band 4 (n + 1) - 1 of large meshes; in-place (substructured) solves only.
constexpr int kWideVariant = 10;
// Separator "variant" that solves with the dense diagonal-block inverses instead of a band
// substitution (tuning caches store it like a band-solve variant).
constexpr int kDenseSep = 100;
extern const BandVariant kBandVariants[kBandVariantCount];
size_t band_variant_smem(int v, bool fp64, int b);
bool band_variant_ok(int v, bool fp64, int b);          // usable by the natural-order block solves
bool band_variant_inplace_ok(int v, bool fp64, int b);  // usable by the in-place (substructured) solves
int band_variant_default(bool fp64, int b);
template <typename T> float time_band_pair(biot_ctx* ctx, bool u, int variant, const T* vin, T* z, int ncols);
// Build the compact diagonal-block inverses a TMA variant needs (no-op if present).
biot_status ensure_dnb(biot_ctx* ctx, bool fp64, bool u, int variant);
biot_status band_setup(biot_ctx* ctx, int kind);
// z = P^{-1} (vin ./ d) for columns [c0, c0 + ncols); vin, z in [n_dof][wcap].
template <typename T> void precond_apply(biot_ctx* ctx, const T* vin, T* z, int c0, int ncols);

// ---- krylov.cu ----
enum ColScalar { CS_RR = 0, CS_BB, CS_BETA0, CS_WN0, CS_WW, CS_INVH, CS_ACTIVE, kColScalars };
// out[s][c] = sum over nblocks per-block partials (fixed order), s < nslots.
void reduce_partials(biot_ctx* ctx, int nslots, int ncols, double* out, int ldo, int c0, int nblocks = kRedBlocks);
template <typename T> biot_status fgmres_cycle(biot_ctx* ctx, int lo, int c0, int ncols);

// ---- batched launches (batch.cu drives them) ----
void launch_batched_residual(const InstDev* tab, int count, cudaStream_t s);
void launch_batched_spmm(const InstDev* tab, int count, bool bf16, int j, cudaStream_t s);
void launch_batched_coupling(const InstDev* tab, int count, int j, cudaStream_t s);
size_t batched_solve_smem(int max_band);  // dynamic shared memory of the batched band solve
biot_status ensure_batch_dnb(biot_ctx* ctx);  // FP32 block inverses in the batched solve's block size
void batched_precond_apply(const InstDev* tab, int count, int j, int max_wcap, int max_band, bool tri,
                           cudaStream_t s);
struct GmgBatch;  // multigrid block solves of a batch (gmg.cu)
void batched_fgmres_cycle(const InstDev* tab, int count, int n_iter, int max_wcap, int max_ndof, int max_band,
                          bool bf16, bool tri, cudaStream_t s, GmgBatch* gb = nullptr);
InstDev inst_describe(biot_ctx* c);
// Batched multigrid: tables of every instance's levels (all contexts set up with multigrid block
// solves, the same smoothing steps, one cycle); update copies the instances' windows to the
// coarse-level table (host) and uploads it; apply replaces batched_precond_apply.
biot_status gmg_batch_create(biot_ctx* const* ctxs, int count, cudaStream_t s, GmgBatch** out);
cudaError_t gmg_batch_update(GmgBatch* gb, const InstDev* tab_h, cudaStream_t s);
void gmg_batch_apply(GmgBatch* gb, const InstDev* tab, int count, int j, bool tri, cudaStream_t s);
void gmg_batch_free(GmgBatch* gb);
bool gmg_batchable(const biot_ctx* c, const biot_ctx* c0);  // same multigrid parameters as c0, one cycle
void batched_residual_reduce(const InstDev* tab, int count, int max_wcap, cudaStream_t s);
biot_status fst_norm2_ctx(biot_ctx* ctx, double* out);
biot_status spacetime_residual_ctx(biot_ctx* ctx, double* out);

}  // namespace biot
