// Batched solve of many independent Biot instances (biot_batch_solve).
//
// Instances of uneven mesh size, permeability field and N_t are solved together:
// every kernel of a sweep (FP64 true residual, FP32 band solves, coupling, AA z,
// CGS2, Givens, FP64 update) processes all instances in one launch, the instance
// given by blockIdx.z and its buffers and window by a device-resident table. Host
// decisions (retiring converged steps, moving windows) are taken once per sweep
// for all instances together; the FGMRES cycle of a sweep has a launch sequence
// that depends only on n_iter, so it is captured once in a CUDA graph and
// replayed every sweep after the table is refreshed. There is no persistent
// kernel and no device-wide wait.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace biot {
namespace {

// out[z][s][c] = colscal_z[(CS_RR + s) * wcap + c] for s < 2, c < wmax (zeros past the window).
__global__ void kb_gather(const InstDev* __restrict__ tab, int wmax, int nslot, double* __restrict__ out) {
  const InstDev& I = tab[blockIdx.z];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (c >= wmax || s >= nslot) return;
  out[((size_t)blockIdx.z * nslot + s) * wmax + c] =
      (I.active && c < I.wcap) ? I.colscal[(size_t)(CS_RR + s) * I.wcap + c] : 0.0;
}

struct BatchState {
  int lo = 1, w = 0;
  bool done = false;
  double rel = INFINITY;
  biot_status st = BIOT_OK;
};

}  // namespace

// The batched kernels' view of one context (FP32 sweep buffers and factors).
InstDev inst_describe(biot_ctx* c) {
  InstDev I{};
  I.n_nodes = c->n_nodes;
  I.n_dof = c->n_dof;
  I.ldx = c->ldx;
  I.wcap = c->wcap;
  I.n_t = c->n_t;
  I.band_u = c->band_u;
  I.band_p = c->band_p;
  I.nodeptr = c->nodeptr;
  I.nbr = c->nbr;
  I.rowptr = c->rowptr;
  I.dsc = c->dsc;
  I.val64 = c->val;
  I.apval64 = c->apval;
  I.X64 = c->X;
  I.F64 = c->F;
  I.X64w = c->X;
  I.val = c->lp.val;
  I.apval = c->lp.apval;
  I.valbf = c->lp.val_bf16;
  I.apvalbf = c->lp.apval_bf16;
  I.V = c->lp.V;
  I.Z = c->lp.Z;
  I.Wv = c->lp.Wv;
  I.tu = c->lp.tu;
  I.tp = c->lp.tp;
  I.Lu = c->lp.Lu;
  I.Uu = c->lp.Uu;
  I.Du = c->lp.Du;
  I.Lp = c->lp.Lp;
  I.Up = c->lp.Up;
  I.Dp = c->lp.Dp;
  I.dsq = c->dsq;
  I.dnbu = c->lp.bdnb[0];
  I.dnbp = c->lp.bdnb[1];
  I.status = c->status;
  I.part = c->part;
  I.colscal = c->colscal;
  I.H = c->H;
  I.hvec = c->hvec;
  I.kcol = c->kcol;
  return I;
}

}  // namespace biot

using namespace biot;

extern "C" biot_status biot_batch_solve(biot_ctx* const* ctxs, int32_t count, double tol, int32_t max_outer,
                                        int32_t use_graph, int32_t* sweeps_done, double* final_rel_res) {
  if (!ctxs || count < 1) return fail(nullptr, BIOT_E_INVALID, "biot_batch_solve: no contexts");
  if (!(tol >= 0.0) || max_outer < 1) return fail(nullptr, BIOT_E_INVALID, "biot_batch_solve: tol >= 0, max_outer >= 1");
  biot_ctx* c0 = ctxs[0];
  for (int i = 0; i < count; ++i) {
    biot_ctx* c = ctxs[i];
    if (!c) return fail(nullptr, BIOT_E_INVALID, "biot_batch_solve: context %d is NULL", i);
    if (!c->assembled || c->precond == 0)
      return fail(c, BIOT_E_STATE, "biot_batch_solve: context %d not assembled and set up", i);
    if (c->prm.precision == BIOT_FP64)
      return fail(c, BIOT_E_INVALID, "biot_batch_solve: context %d must use BIOT_FP32 or BIOT_BF16VAL_FP32ACC", i);
    if (c->prm.precision != c0->prm.precision || c->n_iter != c0->n_iter || c->precond != c0->precond)
      return fail(c, BIOT_E_INVALID, "biot_batch_solve: contexts differ in precision, n_iter or preconditioner");
    if (c->wcap != c->n_t) return fail(c, BIOT_E_INVALID, "biot_batch_solve: context %d needs window = N_t", i);
    if (c0->gmg) {
      if (!gmg_batchable(c, c0))
        return fail(c, BIOT_E_INVALID, "biot_batch_solve: context %d: every context needs multigrid block solves "
                    "with the same smoothing steps and one cycle", i);
    } else if (!c->plain_band || c->gmg) {
      return fail(c, BIOT_E_INVALID, "biot_batch_solve: context %d has no natural-order band factors (n > 512, or "
                  "multigrid block solves mixed with exact ones)", i);
    }
  }
  const bool use_gmg = c0->gmg != nullptr;
  const bool bf16 = c0->prm.precision == BIOT_BF16VAL_FP32ACC;
  const bool tri = c0->precond == BIOT_PRECOND_TRI;
  const int n_iter = c0->n_iter;
  int max_wcap = 0, max_ndof = 0, max_band = 0;
  for (int i = 0; i < count; ++i) {
    max_wcap = std::max(max_wcap, ctxs[i]->wcap);
    max_ndof = std::max(max_ndof, ctxs[i]->n_dof);
    max_band = std::max(max_band, std::max(ctxs[i]->band_u, ctxs[i]->band_p));
  }
  if (!use_gmg && batched_solve_smem(max_band) > 227 * 1024)
    return fail(c0, BIOT_E_INVALID, "biot_batch_solve: half-band %d too wide for the batched band solve", max_band);
  for (int i = 0; i < count; ++i) {
    if (!use_gmg) BIOT_TRY(ensure_batch_dnb(ctxs[i]));
    BIOT_CU(ctxs[i], cudaStreamSynchronize(ctxs[i]->stream));
  }

  cudaStream_t s = nullptr;
  InstDev* tab_d = nullptr;
  InstDev* tab_h = nullptr;
  double* gat_d = nullptr;
  double* gat_h = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  size_t graph_nodes = 0;
  biot_status result = BIOT_OK;
  std::vector<BatchState> B(count);
  GmgBatch* gb = nullptr;
  auto cleanup = [&]() {
    if (gb) gmg_batch_free(gb);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (s) cudaStreamSynchronize(s);
    if (tab_d) cudaFree(tab_d);
    if (gat_d) cudaFree(gat_d);
    if (tab_h) cudaFreeHost(tab_h);
    if (gat_h) cudaFreeHost(gat_h);
    if (s) cudaStreamDestroy(s);
  };
#define BATCH_CU(call)                                                                 \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      result = fail(c0, BIOT_E_CUDA, "biot_batch_solve: %s: %s", #call, cudaGetErrorString(_e)); \
      cleanup();                                                                       \
      return result;                                                                   \
    }                                                                                  \
  } while (0)

  BATCH_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  BATCH_CU(cudaMalloc(&tab_d, sizeof(InstDev) * count));
  BATCH_CU(cudaMalloc(&gat_d, sizeof(double) * count * 2 * max_wcap));
  BATCH_CU(cudaMallocHost(&tab_h, sizeof(InstDev) * count));
  BATCH_CU(cudaMallocHost(&gat_h, sizeof(double) * count * 2 * max_wcap));
  for (int i = 0; i < count; ++i) tab_h[i] = inst_describe(ctxs[i]);
  if (use_gmg) {
    biot_status gst = gmg_batch_create(ctxs, count, s, &gb);
    if (gst != BIOT_OK) {
      cleanup();
      return gst;
    }
  }
  auto upload = [&]() { return cudaMemcpyAsync(tab_d, tab_h, sizeof(InstDev) * count, cudaMemcpyHostToDevice, s); };
  auto gather = [&](int nslot) -> cudaError_t {
    BIOT_LAUNCH(kb_gather, dim3(div_up(max_wcap, 128), nslot, count), 128, 0, s, tab_d, max_wcap, nslot, gat_d);
    cudaError_t e = cudaMemcpyAsync(gat_h, gat_d, sizeof(double) * count * nslot * max_wcap,
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
  };
  auto run_cycle = [&]() -> cudaError_t {
    if (!use_graph) {
      batched_fgmres_cycle(tab_d, count, n_iter, max_wcap, max_ndof, max_band, bf16, tri, s, gb);
      return cudaGetLastError();
    }
    if (!exec) {
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      const int64_t before = g_launches.load();
      batched_fgmres_cycle(tab_d, count, n_iter, max_wcap, max_ndof, max_band, bf16, tri, s, gb);
      g_launches.store(before);  // captured, not launched
      e = cudaStreamEndCapture(s, &graph);
      if (e != cudaSuccess) return e;
      e = cudaGraphInstantiate(&exec, graph, 0);
      if (e != cudaSuccess) return e;
      cudaGraphGetNodes(graph, nullptr, &graph_nodes);
    }
    g_launches.fetch_add((int64_t)graph_nodes);
    return cudaGraphLaunch(exec, s);
  };

  // Tol-schedule sweeps of all instances in lock step (reading A5 per instance):
  // FP64 true residual of every active window, retirement test in FP64, then one
  // FP32 FGMRES cycle per active step whose correction is added to the FP64 state.
  for (;;) {
    bool any = false;
    for (int i = 0; i < count; ++i) {
      BatchState& S = B[i];
      InstDev& I = tab_h[i];
      I.active = 0;
      I.nres = I.nf = 0;
      if (S.done) continue;
      if (S.lo > ctxs[i]->n_t) {
        S.done = true;
        continue;
      }
      if (S.w >= max_outer) {
        S.done = true;
        S.st = BIOT_E_NOT_CONVERGED;
        continue;
      }
      ++S.w;
      // causal start (step n active from sweep n) or, for the eager schedule, every step at once
      const int top = ctxs[i]->prm.schedule == BIOT_SCHED_EAGER ? ctxs[i]->n_t : std::min(S.w, ctxs[i]->n_t);
      const int hi = std::min(top, S.lo + I.wcap - 1);
      I.active = 1;
      I.lo = S.lo;
      I.nres = hi - S.lo + 1;
      any = true;
    }
    if (!any) break;
    BATCH_CU(upload());
    launch_batched_residual(tab_d, count, s);
    batched_residual_reduce(tab_d, count, max_wcap, s);
    BATCH_CU(cudaGetLastError());
    BATCH_CU(gather(2));
    for (int i = 0; i < count; ++i) {
      InstDev& I = tab_h[i];
      if (!I.active) continue;
      BatchState& S = B[i];
      const double* rr = gat_h + ((size_t)i * 2) * max_wcap;
      const double* bb = rr + max_wcap;
      int k = 0;
      while (k < I.nres) {
        const double r = std::sqrt(rr[k]), q = std::sqrt(bb[k]);
        const double rel = q > 0.0 ? r / q : (r == 0.0 ? 0.0 : INFINITY);
        if (!std::isfinite(rel)) {
          S.st = BIOT_E_DIVERGED;
          S.done = true;
          break;
        }
        if (rel <= tol) ++k;
        else break;
      }
      if (S.done) {
        I.active = 0;
        continue;
      }
      I.c0 = k;
      I.nf = I.nres - k;
      S.lo += k;
    }
    BATCH_CU(upload());
    if (gb) BATCH_CU(gmg_batch_update(gb, tab_h, s));
    BATCH_CU(run_cycle());
  }
  BATCH_CU(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) {
    if (final_rel_res) {
      biot_status st = spacetime_residual_ctx(ctxs[i], &B[i].rel);
      if (st != BIOT_OK) {
        cleanup();
        return st;
      }
      final_rel_res[i] = B[i].rel;
    }
    if (sweeps_done) sweeps_done[i] = B[i].w;
    if (B[i].st != BIOT_OK && result == BIOT_OK) {
      result = fail(ctxs[i], B[i].st, "biot_batch_solve: instance %d ended with residual %.3g", i, B[i].rel);
      fail(nullptr, B[i].st, "biot_batch_solve: instance %d ended with residual %.3g", i, B[i].rel);
    }
  }
  cleanup();
#undef BATCH_CU
  return result;
}
