"""Benchmark of the parallel-in-time Biot sweep on GB300.

Workload: the 256x256 Terzaghi column (66,049 nodes, 198,147 DOF), N_t = 256,
tau = 1e-3, E = 1e4, nu = 0.3, alpha = 1, kappa = 1e-6, stabilised P1-P1,
block-diagonal preconditioner P2, FGMRES(10) per step, FP64 (synthetic inputs
shaped like the paper's test cases; see workloads/).

One step = one outer iteration of the inverted time stepping (Alg. 3) over all
N_t = 256 time steps at once: the fused window residual, one preconditioned
FGMRES(10) cycle per time step (10 exact P2 applications by band triangular
solves, 10 AA z products, CGS2) and the convergence norms. This is the work of
one wave of the paper's N_thread = 256 threads.

metric: DOF x timesteps x outer-iterations per second = n_dof * 256 / t_step,
summed over replicas (one independent replica per GPU; the method has no
exchange between independent solves).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF*timesteps*outer-iters/s"
UNIT = "DOF*timesteps*outer-iters/s"
DENSE_SEP = 100   # tuning's separator variant for the dense-block solves
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz
GMG = {"levels": 0, "cycles": 1, "smooth": 2}       # multigrid block solves: automatic depth, V(2, 2)


_SIZE = {}


def workload():
    import workloads as W
    case = W.terzaghi_256("diag")
    if _SIZE:
        case = case.with_(n=_SIZE.get("n", case.n), n_t=_SIZE.get("n_t", case.n_t),
                          name=f"terzaghi_{_SIZE.get('n', case.n)}x{_SIZE.get('n', case.n)}_nt{_SIZE.get('n_t', case.n_t)}")
    return case


def config_dict(case, window):
    return {
        "workload": f"{case.name} (Terzaghi column, stabilised P1-P1, P2 block-diagonal preconditioner)",
        "n": case.n, "n_dof": case.n_dof, "n_t": case.n_t, "tau": case.tau, "E": case.E, "nu": case.nu,
        "kappa": case.kappa, "precond": "P2", "n_iter": case.n_iter, "window": window,
        "step": "one outer iteration (sweep) over all N_t time steps",
        "l2": "no flush: working set ~12 GB >> 126 MB L2 (inputs larger than L2)",
    }


# ---------------------------------------------------------------------------
# CPU oracle sample (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(case, budget_s, max_cols):
    """Time oracle FGMRES(n_iter) cycles (exact LU block solves) on the first time
    steps of a full-window sweep from the zero initial guess. Setup is untimed."""
    import numpy as np
    from oracle.solvers import BlockPreconditioner, fgmres_cycle, step_residual
    from oracle.system import build_system
    s = build_system(case)
    P = BlockPreconditioner(s, case.precond)
    d = s.dscale()
    X = np.zeros((case.n_t + 1, s.n_dof))
    X[0] = s.x0
    times = []
    t_start = time.perf_counter()
    for n in range(1, min(case.n_t, max_cols) + 1):
        t0 = time.perf_counter()
        r, b = step_residual(s, X, n)
        fgmres_cycle(s.AA, P, d, X[n], b, case.n_iter, r=r)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s:
            break
    return s.n_dof, times


def cpu_baseline_subprocess(budget_s=15.0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(budget_s)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        m = re.search(r"^Model name:\s*(.+)$", out, re.M)
        model = m.group(1).strip() if m else None
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        m = re.search(r"^(model name|CPU part)\s*:\s*(.+)$", open("/proc/cpuinfo").read(), re.M)
        model = m.group(2).strip() if m else None
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": os.uname().machine}


def seq_solve_sample(case, max_steps):
    """The sequential baseline (Alg. 1 with an exact solve, as the oracle's seq_solve): sparse LU
    of the equilibrated step matrix factored once, then per step b = A' x_{n-1} + f^n, one solve
    and two FP64 refinement steps. Times the factorisation and the first max_steps steps; the
    full-horizon time is factorisation + N_t x the median step time (every step costs the same)."""
    import numpy as np
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle.system import build_system
    steps = min(case.n_t, max_steps)
    s = build_system(case.with_(n_t=steps))
    d = s.dscale()
    Dm = sp.diags(d)
    t0 = time.perf_counter()
    lu = spla.splu((Dm @ s.AA @ Dm).tocsc())
    t_factor = time.perf_counter() - t0
    x = s.x0.copy()
    times = []
    for n in range(1, steps + 1):
        t0 = time.perf_counter()
        b = s.Ap @ x + s.F[n]
        y = d * lu.solve(d * b)
        for _ in range(2):
            y = y + d * lu.solve(d * (b - s.AA @ y))
        x = y
        times.append(time.perf_counter() - t0)
    per = float(np.median(times))
    full = t_factor + case.n_t * per
    return {"workload": case.name, "n_dof": case.n_dof, "n_t": case.n_t, "factor_s": t_factor,
            "s_per_step": per, "steps_timed": steps, "time_to_solution_s": full,
            "extrapolated": steps < case.n_t, "dof_steps_per_s": case.n_dof * case.n_t / full}


def run_cpu_sample(budget_s):
    import workloads as W
    case = workload()
    n_dof, times = oracle_sample(case, budget_s, case.n_t)
    tot = sum(times)
    seq = {"small": seq_solve_sample(W.terzaghi_small(), 10 ** 9), "bench": seq_solve_sample(case, 8)}
    print(json.dumps({
        "value": n_dof * len(times) / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": f"{len(times)} of the {case.n_t} time steps of one full-window sweep at {case.n}x{case.n} "
                  f"(oracle FGMRES({case.n_iter}) cycles with exact sparse-LU block solves, single thread, "
                  f"{tot:.1f} s timed; assembly and factorisation untimed)",
        "host": host_cpu(),
        "seq_solve": seq,
        "seq_solve_note": "sequential backward Euler (sparse LU factored once, N_t exact step solves) on one "
                          "core: the time to solution of the method the paper parallelises; 'bench' times the "
                          "factorisation and 8 of the 256 steps and extrapolates",
    }))


# ---------------------------------------------------------------------------
# distributed helpers (one independent replica per GPU)
# ---------------------------------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------

def strip_envelope(w, C, d):
    """Off-diagonal entries of the Cholesky factor of one strip interior: the strip's nodes in
    order (rows j outer, its w node columns inner), d fields each; row r of node (ii, j) reaches
    back to the first field of its lowest-numbered neighbour among (ii - 1, j - 1), (ii, j - 1),
    (ii - 1, j) and itself (the "/"-split mesh), and a factor fills its matrix's row envelope.
    At most the half-band d (w + 2) - 1 that the band kernels sweep (the rows of a strip's first
    node column and its first node row reach back less)."""
    import numpy as np
    j, ii = np.meshgrid(np.arange(C), np.arange(w), indexing="ij")
    node = j * w + ii
    low = node.copy()
    low = np.where(ii >= 1, node - 1, low)                        # (ii - 1, j)
    low = np.where(j >= 1, (j - 1) * w + ii, low)                 # (ii, j - 1)
    low = np.where((j >= 1) & (ii >= 1), (j - 1) * w + ii - 1, low)  # (ii - 1, j - 1)
    back = d * (node - low)                                       # field 0 of the node
    return float(sum(back.sum() + f * back.size for f in range(d)))


def band_solve_flops(info, ncols, precond, strips=0, dense_sep=(True, True)):
    """Algorithmic FP64 flops of the exact block solves of one P apply: 2 flops per structurally
    nonzero off-diagonal factor entry per column of every triangular solve.

    Plain band factors (strips < 2): forward + backward on A (half-band 2n+5) and on S
    (n+2), tri(N, b) = 2 W (N b - b (b + 1) / 2). Substructured (strips >= 2, the library's
    layout): per block (d = 2 for A, 1 for S) two forward + backward pairs on every strip
    interior (its factor's row envelope, strip_envelope) and one pair on the separators' Schur
    complement, whose factor is block bidiagonal with B = d (n + 1): a dense lower triangle per
    block and a dense B x B block below it for every block but the first (the rest of its
    half-band 2B - 1 is exact zeros, skipped by the solves), plus the two sparse couplings (2 flops
    per separator-interior entry per column, twice: each separator node has four interior
    neighbours, two fewer on the first and last node rows). The dense-block separator solves
    (dense_sep[block]) do the same multiply-adds (block-diagonal products with the inverted
    diagonal blocks: B (B - 1) / 2 per block; chain products: B^2 per block but the first).
    Also returns the launches of one apply."""
    def tri(N, b):
        return 2.0 * ncols * (N * b - b * (b + 1) / 2.0)
    n = round((info.n_nodes) ** 0.5) - 1
    if strips < 2:
        fa = tri(2 * info.n_nodes, info.band_u)
        fs = tri(info.n_nodes, info.band_p)
        return 2 * fa + 2 * fs, 4
    C = n + 1
    ni = C - (strips - 1)
    widths = [ni // strips + (1 if t < ni % strips else 0) for t in range(strips)]
    total = 0.0
    launches = 0
    for blk, d in enumerate((2, 1)):
        interior = 2.0 * ncols * sum(strip_envelope(w, C, d) for w in widths)
        B, nb = d * C, strips - 1
        sep = 2.0 * ncols * (B * (B - 1) / 2.0 + (nb - 1) * (B * B + B * (B - 1) / 2.0))
        coupling = 2 * 2.0 * ncols * nb * (4 * C - 2) * d * d
        total += 4 * interior + 2 * sep + coupling
        # gather, 2 x interior pair, 2 couplings, scatter; separators: a pair of band solves,
        # or two block-diagonal products and two chains of nb - 1 products
        launches += 8 + (2 * nb if dense_sep[blk] else 2)
    return total, launches


def sweep_bytes(info, ncols, n_iter, precision, precond, strips=0, dense_sep=(True, True), gmg=None):
    """Algorithmic DRAM bytes of one sweep over ncols active steps, by kernel class: every
    matrix entry, factor entry and vector element a kernel must read or write, once.

    s = 8 (FP64) or 4 (FP32 / BF16-value sweeps: Krylov vectors, factors and workspaces in FP32;
    s_v = 2 for the BF16 SpMM values). Per sweep:
      residual  (always FP64, output V_0 in s): nnz*12 + P*8 + 4(N+1) + N W (8 + 8 + s) + 8 N
      per Arnoldi step j = 0 .. n_iter - 1:
        P apply   per block (A: d = 2, S: d = 1; N_b = d (n+1)^2 rows, N_S = d (k-1)(n+1) separator
                  rows, N_I = N_b - N_S): gather and scatter 4 N_b W s; four interior solves (two
                  forward + backward pairs) 4 (E_I s + 2 N_I W s) with E_I the factor entries
                  (diagonal included); two couplings 2 (2 N_S + 2 N_S) W s; separators: dense
                  blocks E_S s (lower triangles of the k - 1 inverted diagonal blocks twice, the
                  k - 2 products M_K and P_K) plus 4 passes 2 N_S W s over the workspace.
                  (Plain band factors: four solves reading the factor and 2 N_b W s each.)
                  P1 adds the coupling B^T z_u: 4 P s_v + 2 n_nodes W s + n_nodes W s.
        SpMM      nnz (s_v + 4) + 4 (N+1) + 2 N W s
        CGS2      two passes of dots ((j+1) + ceil((j+1)/8)) N W s and Gram-Schmidt update
                  (j+1+2) N W s, one norm N W s, one column scaling 2 N W s (not after the last).
                  FP32 / BF16 sweeps: the norm rides on the second update, and up to 12 basis
                  vectors the first update also forms the second sweep's dots (no second dots
                  pass)
      update      n_iter N W s (Z) + 2 N W 8 (X in FP64) and the initial scaling 2 N W s
    """
    import math
    N, nn, nnz, P, W = info.n_dof, info.n_nodes, info.nnz, info.n_pairs, ncols
    fp64 = precision == "fp64"
    s = 8 if fp64 else 4
    s_v = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    n = round(nn ** 0.5) - 1
    C = n + 1
    out = {"residual": nnz * 12 + P * 8 + 4 * (N + 1) + N * W * (8 + 8 + s) + 8 * N}
    apply_b = 0.0
    for blk, d in enumerate((2, 1)):
        Nb = d * nn
        if strips < 2:
            b = info.band_u if d == 2 else info.band_p
            entries = Nb * (b + 1) - b * (b + 1) / 2.0
            apply_b += 2 * (entries * s + 2 * Nb * W * s)
            continue
        ni = C - (strips - 1)
        widths = [ni // strips + (1 if t < ni % strips else 0) for t in range(strips)]
        nb = strips - 1
        NS = d * nb * C
        NI = Nb - NS
        EI = sum(strip_envelope(w, C, d) for w in widths) + NI
        B = d * C
        ES = 2 * nb * B * (B + 1) / 2.0 + 2 * max(nb - 1, 0) * B * B
        apply_b += 4 * Nb * W * s + 4 * (EI * s + 2 * NI * W * s) + 2 * 4 * NS * W * s
        apply_b += ES * s + 4 * 2 * NS * W * s
    if precond == "tri":
        apply_b += 4 * P * s_v + 3 * nn * W * s
    if gmg is not None:  # multigrid block solves replace the factorisations
        apply_b = gmg_apply_bytes(n, (W + 3) // 4 * 4, s, precond, gmg.get("smooth", 2), gmg.get("cycles", 1),
                                  gmg.get("levels", 0))
    out["block_solves"] = n_iter * apply_b
    out["spmm"] = n_iter * (nnz * (s_v + 4) + 4 * (N + 1) + 2 * N * W * s)
    kry = 2 * N * W * s + n_iter * N * W * s + 2 * N * W * 8
    for j in range(n_iter):
        dots = ((j + 1) + math.ceil((j + 1) / 8)) * N * W * s
        upd = (j + 3) * N * W * s
        if fp64:
            kry += 2 * (dots + upd) + N * W * s
        else:
            kry += dots + 2 * upd + (dots if j + 1 > 12 else 0)
        kry += 2 * N * W * s if j + 1 < n_iter else 0
    out["krylov"] = kry
    out["total"] = sum(out.values())
    out["per_apply_block_solves"] = apply_b
    return out


def gmg_levels(n, req=0):
    """Levels of the library's multigrid hierarchy (automatic: halve while n is even and > 16)."""
    L, m = 1, n
    while m % 2 == 0 and (m > 16 if req <= 0 else (m // 2 >= 2 and L < req)):
        m //= 2
        L += 1
    return L


def gmg_apply_bytes(n, W, s, precond, smooth=2, cycles=1, levels=0):
    """Algorithmic DRAM bytes of one P apply with multigrid block solves (biot_set_inner_solver).

    Per level l < L-1 (R = rows of the fields in the cycle, VB = R W s one vector pass): the first
    smoothing step from zero 2 VB (b in, x out: its increment is x, where the next step reads it),
    every other step x and b in, x out, the increment d in unless the previous step started from
    zero, d out unless it is the smoothing's last step (the 7-point stencil's neighbour rows are
    cache hits): 5 VB for the middle steps, residual 3 VB, restriction VB + VB_c,
    prolongation 2 VB + VB_c, and the stencil coefficients (40 values per node) read by each of
    the 2 smooth + 1 passes over the level. Coarsest level: its input 2 VB (the band solves of a
    16^2 mesh are negligible). Level 0 adds the right-hand side (input rows in, b out: 2 VB) and
    the result (x in, z out: 2 VB). P2 runs A's and S's rows in one cycle (3 rows per node); P1
    one cycle on A's rows, the coupling B^T z_u (z_u, tp and 4 values per node pair), one on
    S's. Each extra cycle adds a residual (3 VB) and an update (3 VB) on level 0."""
    L = gmg_levels(n, levels)

    def cycle(rows_per_node):
        tot = 0.0
        for l in range(L):
            nl = n >> l
            nn = (nl + 1) ** 2
            VB = rows_per_node * nn * W * s
            if l == L - 1:
                tot += 2 * VB
                continue
            VBc = rows_per_node * ((nl // 2) + 1) ** 2 * W * s
            for pre in (True, False):
                for k in range(smooth):
                    if pre and k == 0:
                        tot += 2 * VB
                        continue
                    d_in = k > 0 and not (pre and k == 1)
                    d_out = k + 1 < smooth
                    tot += (3 + d_in + d_out) * VB
            tot += 3 * VB + VB + VBc + 2 * VB + VBc      # residual, restriction, prolongation
            tot += (2 * smooth + 1) * nn * 40 * s
        nn0 = (n + 1) ** 2
        VB0 = rows_per_node * nn0 * W * s
        tot += 4 * VB0 + (cycles - 1) * 6 * VB0
        return tot * (1 + (cycles - 1))

    nn0 = (n + 1) ** 2
    if precond == "diag":
        return cycle(3)
    P = 7 * n * n + 6 * n + 1
    return cycle(2) + cycle(1) + 4 * P * s + 3 * nn0 * W * s


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def streaming_kernels(info, ncols, precision, res_ms, res_n, spmm_ms, spmm_n):
    """Algorithmic bytes and achieved bandwidth of the sparse sweep kernels.

    Residual (one CSR pass over AA and A'): nnz*(s_v + 4) + P*s_v + 4*(N_dof + 1)
    + N_dof*W*(s_x [X] + s_x [F] + s_o [R]) + N_dof*s_x [X column lo - 1]; the residual
    is always formed in FP64 (s_v = s_x = 8) and written in the sweep's precision s_o.
    SpMM (w = d .* AA z): the same without F and the extra column, in the sweep's
    precision. Both also carry an FP64 ALU roof: 2*(nnz + P)*W flops for the residual,
    2*nnz*W for the SpMM at the derived FP64 peak (FP32 one for the FP32 SpMM)."""
    hbm, src = _hbm_peak()
    nd, nnz, P = info.n_dof, info.nnz, info.n_pairs
    s_o = 8 if precision == "fp64" else 4
    s_z = 8 if precision == "fp64" else 4
    s_val = {"fp64": 8, "fp32": 4, "bf16": 2}[precision]
    res_bytes = nnz * (8 + 4) + P * 8 + 4 * (nd + 1) + nd * ncols * (8 + 8 + s_o) + nd * 8
    spmm_bytes = nnz * (s_val + 4) + 4 * (nd + 1) + nd * ncols * 2 * s_z
    out = {}
    for name, ms, n, by, flops, alu in (
            ("residual", res_ms, res_n, res_bytes, 2.0 * (nnz + P) * ncols, FP64_PEAK_TFLOPS),
            ("spmm", spmm_ms, spmm_n, spmm_bytes, 2.0 * nnz * ncols,
             FP64_PEAK_TFLOPS if precision == "fp64" else FP32_PEAK_TFLOPS)):
        if not n:
            continue
        t = ms / n / 1e3
        out[name] = {"ms_per_launch": ms / n, "launches": n, "algorithmic_bytes": int(by),
                     "achieved_gbs": by / t / 1e9, "hbm_peak_gbs": hbm, "hbm_frac": by / t / 1e9 / hbm,
                     "peak_source": src, "alu_roof_ms": flops / (alu * 1e12) * 1e3,
                     "alu_frac": flops / t / 1e12 / alu}
    return out


def kernel_source_hash(src_path, kernel):
    """sha256[:16] of one kernel's definition: from the template line above `kernel(`
    at the start of a line to the first closing brace in column 0 after it."""
    txt = open(src_path).read()
    at = txt.find("\n" + kernel + "(")
    if at < 0:
        return None
    start = txt.rfind("\ntemplate <", 0, at)
    start = at if start < 0 else start
    end = txt.find("\n}\n", at)
    return hashlib.sha256(txt[start:end + 3].encode()).hexdigest()[:16]


# The kernels of one P apply's block solves, (source file, definition) pairs.
APPLY_KERNELS = [("band.cu", "k_band_solve_rows"), ("band.cu", "band_solve_tma_body"),
                 ("separator.cu", "k_sep_gemm")]


def dense_sep_of(tuning):
    """Which blocks (A, S) solve their separators with the dense block products."""
    return (tuning.get("variant_sep_u") == DENSE_SEP, tuning.get("variant_sep_p") == DENSE_SEP)


def sources_hash(files):
    """sha256[:16] of whole source files under paper_2310_10430_gb300/csrc, chained in order."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2310_10430_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# The sources of every kernel one reduced-precision sweep launches.
SWEEP_SOURCES = ["band.cu", "gmg.cu", "krylov.cu", "separator.cu", "spmm.cu", "substructure.cu"]


def profile_traffic_sha(sha, unit_tag):
    """DRAM bytes per unit from the committed ncu summary that records this source hash."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, fn)).read()
        m1 = re.search(r"sources_sha256_16:\s*([0-9a-f]{16})", txt)
        m2 = re.search(r"traffic_bytes_per_%s:\s*([0-9.eE+]+)" % unit_tag, txt)
        if m1 and m2 and m1.group(1) == sha:
            return float(m2.group(1))
    return None


def profile_traffic(parts):
    """DRAM bytes per unit from a committed ncu summary whose kernel-source hash matches (null
    once a kernel has changed since the counters were taken): the hashes of the (file,
    definition) parts under paper_2310_10430_gb300/csrc are chained."""
    hs = [kernel_source_hash(os.path.join(ROOT, "paper_2310_10430_gb300", "csrc", f), k) for f, k in parts]
    sha = None if None in hs else hashlib.sha256("".join(hs).encode()).hexdigest()[:16]
    pdir = os.path.join(ROOT, "profiles")
    if sha is None or not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, fn)).read()
        m1 = re.search(r"source_sha256_16:\s*([0-9a-f]{16})", txt)
        m2 = re.search(r"traffic_bytes_per_unit:\s*([0-9.eE+]+)", txt)
        if m1 and m2 and m1.group(1) == sha:
            return float(m2.group(1))
    return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    from paper_2310_10430_gb300 import biot
    from paper_2310_10430_gb300 import build as B

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    barrier(world)
    if rank != 0:
        B.build()
    case = workload()
    stream = torch.cuda.current_stream()
    W_ = case.n_t
    ctx = biot.Context(case, stream=stream, window=W_, precision=args.precision, strips=args.strips,
                       gmg=GMG if args.gmg else None)
    info = ctx.info
    lo, hi = 1, case.n_t
    tuning = biot.biot_tune(ctx.ctx, args.tune_cache).as_dict()

    for _ in range(args.warmup):
        biot.biot_sweep(ctx.ctx, lo, hi, want_rel=False)
    torch.cuda.synchronize()

    # ---- device-timed region -------------------------------------------------
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    biot.biot_timing_enable(ctx.ctx, True)
    l0 = biot.biot_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nvtx_push("timed_sweeps")  # lets a profiler's launch list select exactly the timed region
    e0.record(stream)
    for _ in range(args.steps):
        biot.biot_sweep(ctx.ctx, lo, hi, want_rel=False)
    e1.record(stream)
    nvtx_pop()
    torch.cuda.synchronize()
    launches = biot.biot_launch_count() - l0 - 0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    band_ms, band_n = biot.biot_timing_read(ctx.ctx, biot.BIOT_KC_BAND_SOLVE)
    res_ms, res_n = biot.biot_timing_read(ctx.ctx, biot.BIOT_KC_RESIDUAL)
    spmm_ms, spmm_n = biot.biot_timing_read(ctx.ctx, biot.BIOT_KC_SPMM)
    biot.biot_timing_enable(ctx.ctx, False)
    barrier(world)
    ms_max = allreduce_max(ms, world)
    ms_per_step = ms_max / args.steps
    units_per_step = case.n_dof * (hi - lo + 1)
    value = world * units_per_step / (ms_per_step / 1e3)

    # ---- end to end through the C ABI with pinned host buffers --------------
    nd = case.n_dof
    host_in = torch.empty((hi + 1, nd), dtype=torch.float64, pin_memory=True).numpy()
    host_out = torch.empty((hi - lo + 1, nd), dtype=torch.float64, pin_memory=True).numpy()
    biot.biot_get_state(ctx.ctx, 0, hi, host_in)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        biot.biot_set_state(ctx.ctx, 0, hi, host_in)
        rel = biot.biot_sweep(ctx.ctx, lo, hi, want_rel=True)
        biot.biot_get_state(ctx.ctx, lo, hi, host_out)
    torch.cuda.synchronize()
    e2e_s = allreduce_max(time.perf_counter() - t0, world) / args.steps
    e2e_value = world * units_per_step / e2e_s
    h2d = host_in.nbytes
    d2h = host_out.nbytes + rel.nbytes

    # ---- roofline of the dominant kernel (band triangular solves, FP64 ALU) --
    # the band-solve timing class brackets one whole P apply (its four solve launches; for
    # P2 the solves on A and on S run concurrently on two streams)
    flops_per_apply, launches_per_apply = band_solve_flops(info, hi - lo + 1, case.precond,
                                                           int(tuning.get("strips", 0)), dense_sep_of(tuning))
    achieved = flops_per_apply / (band_ms / band_n / 1e3) / 1e12
    traffic = profile_traffic(APPLY_KERNELS) if args.precision == "fp64" else None
    fp64 = args.precision == "fp64"
    peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
    roofline = {"kernel": "k_band_solve_rows + k_sep_gemm + k_band_solve_tma (%s exact block solves of the P2 "
                          "apply: strip interiors, dense-block and band separator solves)" % ("FP64" if fp64 else "FP32"),
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "peak_source": ("derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz (FP64 not in MEASURED_PEAKS.json)"
                                if fp64 else "derived: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz"),
                "traffic": traffic, "traffic_per": "P apply (DRAM bytes of its band-solve and separator launches)",
                "applies": band_n, "launches_per_apply": launches_per_apply,
                "avg_apply_ms": band_ms / band_n, "avg_launch_ms": band_ms / band_n / launches_per_apply,
                "share_of_step": band_ms / ms}
    if args.gmg:
        # multigrid block solves (profiling runs): the V-cycle apply against HBM
        hbm, src = _hbm_peak()
        s_el = 8 if fp64 else 4
        by_apply = gmg_apply_bytes(case.n, (W_ + 3) // 4 * 4, s_el, case.precond, GMG["smooth"], GMG["cycles"],
                                   GMG["levels"])
        ach = by_apply / (band_ms / band_n / 1e3) / 1e9
        roofline = {"kernel": "k_gmg_* (multigrid V-cycle apply of P2: smoothing, residual, transfers, coarsest "
                              "band solve)", "bound": "hbm", "achieved": ach, "peak": hbm, "peak_source": src,
                    "unit": "GB/s", "frac": ach / hbm, "traffic": None, "traffic_per": "P apply",
                    "bytes_per_apply": by_apply, "applies": band_n, "avg_apply_ms": band_ms / band_n,
                    "share_of_step": band_ms / ms}

    streaming = streaming_kernels(info, hi - lo + 1, args.precision, res_ms, res_n, spmm_ms, spmm_n)

    ctx.close()
    extras = {}
    if not args.no_extras:
        extras["variants"] = {p: sweep_variant(case, p, max(2, args.steps // 2), 2, stream) for p in ("fp32", "bf16")}
        for p in ("fp32", "fp64"):
            extras["variants"][p + "_gmg"] = sweep_variant(case, p, max(2, args.steps // 2), 2, stream, gmg=GMG)
        extras["time_to_solution"] = time_to_solution(workload().with_(n=64, n_t=64, name="terzaghi_64x64_nt64"),
                                                      stream)
        extras["batched"] = batched_vs_sequential(stream)
        try:
            extras["batched_config4"] = batched_config4(stream)
        except Exception as e:  # e.g. device memory: report, keep the bench line
            extras["batched_config4"] = {"error": str(e)[:300]}
        if world == 1:
            # the 1024^2 stress workload's sweep with multigrid block solves (94 GB on the device);
            # its time to error is the --large --large-gmg --large-error run
            import types
            try:
                extras["large_1024"] = large_mesh(types.SimpleNamespace(
                    steps=2, warmup=3, large_outer=0, large_gmg=True, large_error=False, large_n_iter=20,
                    large_tols=None, large_ref_gmg=False, strips=None, tune_cache=None), quiet=True)
            except Exception as e:
                extras["large_1024"] = {"error": str(e)[:300]}
    if args.lognormal:
        extras["lognormal_precisions"] = lognormal_precisions(stream, args.lognormal)
    if args.efficiency:
        extras["efficiency"] = efficiency_study(stream)
    if args.barry_mercer:
        extras["barry_mercer"] = barry_mercer_study(stream)
    if args.mandel:
        extras["mandel"] = mandel_study(stream)
    if args.batched_full:
        extras["batched_config4_full"] = batched_config4(stream, full=True)
    out = None
    if rank == 0:
        cpu = cpu_baseline_subprocess(args.cpu_budget) if (world == 1 and not args.no_cpu) else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "f32"}[args.precision],
            "data": "synthetic", "config": config_dict(case, W_),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "kernels_ms_per_step": {"band_solve": band_ms / args.steps, "residual": res_ms / args.steps,
                                    "spmm": spmm_ms / args.steps},
            "streaming_kernels": streaming,
            "cpu_baseline": cpu,
            "tuning": tuning,
        }
        out.update(extras)
        if "variants" in extras:
            # the bandwidth target of the method is the reduced-precision sweep: its HBM roofline,
            # for the multigrid block solves (the streaming form) and for the exact factorisations
            out["roofline_fp32"] = dict(extras["variants"]["fp32_gmg"]["roofline"],
                                        sweep="FP32 sweep of the bench workload (FP64 residual and update), "
                                              "multigrid block solves")
            out["roofline_fp32_exact"] = dict(extras["variants"]["fp32"]["roofline"],
                                              sweep="FP32 sweep of the bench workload, exact block solves")
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------------------
# secondary measurements: reduced-precision sweeps, time to solution, batching
# ---------------------------------------------------------------------------



def sweep_variant(case, precision, steps, warmup, stream, gmg=None):
    """Time reduced-precision sweeps over all N_t steps at the bench workload (FP64 true
    residual, FP32 FGMRES cycle on the correction, FP64 update); returns ms per sweep
    and the band-solve roofline in FP32."""
    import torch
    from paper_2310_10430_gb300 import biot
    with biot.Context(case, stream=stream, precision=precision, gmg=gmg) as c:
        info = c.info
        tuning = biot.biot_tune(c.ctx, None).as_dict()
        for _ in range(warmup):
            biot.biot_sweep(c.ctx, 1, case.n_t, want_rel=False)
        torch.cuda.synchronize()
        biot.biot_timing_enable(c.ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            biot.biot_sweep(c.ctx, 1, case.n_t, want_rel=False)
        e1.record(stream)
        torch.cuda.synchronize()
        band_ms, band_n = biot.biot_timing_read(c.ctx, biot.BIOT_KC_BAND_SOLVE)
        res_ms, res_n = biot.biot_timing_read(c.ctx, biot.BIOT_KC_RESIDUAL)
        spmm_ms, spmm_n = biot.biot_timing_read(c.ctx, biot.BIOT_KC_SPMM)
        biot.biot_timing_enable(c.ctx, False)
        ms = e0.elapsed_time(e1) / steps
        strips = int(tuning.get("strips", 0))
        fl, per = band_solve_flops(info, case.n_t, case.precond, strips, dense_sep_of(tuning))
        ach = fl / (band_ms / band_n / 1e3) / 1e12
        hbm, src = _hbm_peak()
        by = sweep_bytes(info, case.n_t, case.n_iter, precision, case.precond, strips, gmg=gmg)
        apply_ms = band_ms / band_n
        kms = {"band_solve": band_ms / steps, "residual": res_ms / steps, "spmm": spmm_ms / steps}
        kms["krylov_and_rest"] = ms - sum(kms.values())
        return {"ms_per_step": ms, "value": case.n_dof * case.n_t / (ms / 1e3), "unit": UNIT,
                "band_solve": {"achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "bound": "alu",
                               "frac": ach / FP32_PEAK_TFLOPS, "share_of_step": band_ms / steps / ms},
                # the whole sweep against HBM: algorithmic bytes of every kernel class over the sweep time
                "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm, "peak_source": src,
                             # ncu DRAM read + write of one sweep, from the committed summary whose
                             # source hash matches these sources (null once they changed)
                             "traffic": (profile_traffic_sha(sources_hash(SWEEP_SOURCES),
                                                             "gmg_sweep" if gmg else "exact_sweep")
                                         if precision == "fp32" else None),
                             "traffic_per": "one FP32 sweep",
                             "achieved": by["total"] / (ms / 1e3) / 1e9,
                             "frac": by["total"] / (ms / 1e3) / 1e9 / hbm,
                             "algorithmic_bytes_per_sweep": by["total"],
                             "bytes_by_class": {k: by[k] for k in ("residual", "block_solves", "spmm", "krylov")},
                             "time_at_roof_ms": by["total"] / (hbm * 1e9) * 1e3,
                             "block_solves": {"achieved": by["per_apply_block_solves"] / (apply_ms / 1e3) / 1e9,
                                              "frac": by["per_apply_block_solves"] / (apply_ms / 1e3) / 1e9 / hbm,
                                              "bytes_per_apply": by["per_apply_block_solves"],
                                              "avg_apply_ms": apply_ms}},
                "kernels_ms_per_step": kms,
                "block_solves": ("multigrid V-cycles (%d levels, %s)" % (info.gmg_levels, gmg)) if gmg
                                else "exact (substructured factorisations)",
                "tuning": {k: tuning[k] for k in ("variant_u", "variant_p", "nb_u", "threads_u", "tma_u", "strips",
                                                  "variant_sep_u", "variant_sep_p", "spmm_variant", "ms_spmm",
                                                  "ms_spmm_default")}}


def time_to_solution(case, stream):
    """Wall time of complete solves (setup excluded) to the same FP64 residual
    tolerance 1e-10: plain FP64 PinT, and the FP32 / BF16-value sweeps with the FP64
    residual and update (refinement per sweep), each checked against a FP64 solve
    converged to 1e-13."""
    import numpy as np
    import torch
    from paper_2310_10430_gb300 import biot
    with biot.Context(case, stream=stream) as c:
        biot.biot_pint_solve(c.ctx, 1e-13, 100000)
        ref = biot.biot_get_state(c.ctx, 1, case.n_t)
    out = {"workload": f"{case.name}: n={case.n}, N_t={case.n_t}, P2, setup (assembly, factorisation) excluded"}
    for prec in ("fp64", "fp32", "bf16"):
        with biot.Context(case, stream=stream, precision=prec) as c:
            biot.biot_tune(c.ctx, None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 100000, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            X = biot.biot_get_state(c.ctx, 1, case.n_t)
        eu = float(np.linalg.norm(X[:, 0::3] - ref[:, 0::3]) ** 2 + np.linalg.norm(X[:, 1::3] - ref[:, 1::3]) ** 2) ** 0.5
        eu /= float(np.linalg.norm(ref[:, 0::3]) ** 2 + np.linalg.norm(ref[:, 1::3]) ** 2) ** 0.5
        ep = float(np.linalg.norm(X[:, 2::3] - ref[:, 2::3]) / np.linalg.norm(ref[:, 2::3]))
        out[prec] = {"seconds": dt, "sweeps": sweeps, "status": biot.STATUS_NAMES[st], "rel_residual": rel,
                     "rel_err_u": eu, "rel_err_p": ep}
    # The paper's own schedule (Alg. 3 with N_thread = M): every step gets exactly M FGMRES
    # cycles while M steps are in flight, N_t + M - 1 sweeps of M columns each; the error
    # against the converged solve decides which M reaches 1e-8.
    # Restart length: the same tolerance solve with longer FGMRES cycles (more Arnoldi steps
    # per sweep, fewer sweeps); the bench's throughput metric stays at n_iter = 10.
    for prec in ("fp64", "fp32"):
        for n_iter in (20, 30):
            cn = case.with_(n_iter=n_iter)
            with biot.Context(cn, stream=stream, precision=prec) as c:
                biot.biot_tune(c.ctx, None)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 100000, allow_not_converged=True)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                X = biot.biot_get_state(c.ctx, 1, case.n_t)
            eu, ep = _field_errors(np, X, ref)
            out[f"{prec}_n_iter{n_iter}"] = {"seconds": dt, "sweeps": sweeps, "status": biot.STATUS_NAMES[st],
                                             "rel_residual": rel, "rel_err_u": eu, "rel_err_p": ep}
    # multigrid block solves (inexact P^{-1}; the flexible cycle converges to the same solution)
    for prec in ("fp64", "fp32"):
        for n_iter in (10, 30):
            cn = case.with_(n_iter=n_iter)
            with biot.Context(cn, stream=stream, precision=prec, gmg=GMG) as c:
                biot.biot_tune(c.ctx, None)   # the SpMM shape
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 100000, allow_not_converged=True)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                X = biot.biot_get_state(c.ctx, 1, case.n_t)
            eu, ep = _field_errors(np, X, ref)
            out[f"{prec}_gmg_n_iter{n_iter}"] = {"seconds": dt, "sweeps": sweeps, "status": biot.STATUS_NAMES[st],
                                                 "rel_residual": rel, "rel_err_u": eu, "rel_err_p": ep}
    paper = {}
    for prec in ("fp64", "fp32"):
        for M in (8, 16):
            with biot.Context(case, stream=stream, precision=prec, window=M, schedule=biot.BIOT_SCHED_PAPER) as c:
                biot.biot_tune(c.ctx, None)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, sweeps, rel = biot.biot_pint_solve(c.ctx, 0.0, 100000, allow_not_converged=True)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                X = biot.biot_get_state(c.ctx, 1, case.n_t)
            eu, ep = _field_errors(np, X, ref)
            paper[f"{prec}_M{M}"] = {"seconds": dt, "sweeps": sweeps, "rel_residual": rel, "rel_err_u": eu,
                                     "rel_err_p": ep}
    out["paper_schedule"] = paper
    ok = {k: v for k, v in paper.items() if max(v["rel_err_u"], v["rel_err_p"]) <= 1e-8}
    tol_ok = {k: out[k]["seconds"] for k in ("fp64", "fp32", "bf16", "fp64_n_iter20", "fp64_n_iter30",
                                             "fp32_n_iter20", "fp32_n_iter30", "fp64_gmg_n_iter10",
                                             "fp64_gmg_n_iter30", "fp32_gmg_n_iter10", "fp32_gmg_n_iter30")
              if max(out[k]["rel_err_u"], out[k]["rel_err_p"]) <= 1e-8}
    cands = {**{f"tol_{k}": v for k, v in tol_ok.items()}, **{f"paper_{k}": v["seconds"] for k, v in ok.items()}}
    if cands:
        best = min(cands, key=cands.get)
        out["fastest_to_1e-8"] = {"run": best, "seconds": cands[best]}
    return out


def _field_errors(np, X, ref):
    eu = float(np.linalg.norm(X[:, 0::3] - ref[:, 0::3]) ** 2 + np.linalg.norm(X[:, 1::3] - ref[:, 1::3]) ** 2) ** 0.5
    eu /= float(np.linalg.norm(ref[:, 0::3]) ** 2 + np.linalg.norm(ref[:, 1::3]) ** 2) ** 0.5
    ep = float(np.linalg.norm(X[:, 2::3] - ref[:, 2::3]) / np.linalg.norm(ref[:, 2::3]))
    return eu, ep


def lognormal_precisions(stream, n_t):
    """The lognormal-permeability workload (256^2, sigma 1, l = 0.1, seed 1234, P1): FP32 and
    BF16-value sweeps with the FP64 residual and update against the FP64 solve, all to the same
    FP64 residual tolerance 1e-10 with FGMRES(30); errors per field against an FP64 solve
    converged to 1e-12. n_t bounds the run time (the full workload has N_t = 256)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2310_10430_gb300 import biot
    case = W.lognormal_256().with_(n_t=n_t, n_iter=30, name=f"lognormal_256x256_nt{n_t}")
    with biot.Context(case, stream=stream) as c:
        biot.biot_tune(c.ctx, None)
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 100000, allow_not_converged=True)
        ref = biot.biot_get_state(c.ctx, 1, case.n_t)
    out = {"workload": f"{case.name}: n=256, N_t={n_t}, lognormal kappa sigma 1, P1, FGMRES(30), "
                       "setup excluded", "reference": {"sweeps": sweeps, "rel_residual": rel,
                                                       "status": biot.STATUS_NAMES[st]}}
    for prec in ("fp64", "fp32", "bf16"):
        with biot.Context(case, stream=stream, precision=prec) as c:
            biot.biot_tune(c.ctx, None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 100000, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            X = biot.biot_get_state(c.ctx, 1, case.n_t)
        eu, ep = _field_errors(np, X, ref)
        out[prec] = {"seconds": dt, "sweeps": sweeps, "status": biot.STATUS_NAMES[st], "rel_residual": rel,
                     "rel_err_u": eu, "rel_err_p": ep}
    return out


def efficiency_study(stream, n=64, n_t=64, Ms=(1, 2, 4, 8, 16, 32, 64)):
    """The paper's parallel-efficiency model (Sec. 3.2, Eqs. e1_theo and E2_theo) measured on the
    GPU, Terzaghi n x n, N_t steps, FGMRES(10) cycles, P2, FP64. For each N_thread = M:
    * inverted time stepping, the paper schedule (Alg. 3 with window M): N_t + M - 1 sweeps of at
      most M columns, every step M cycles (N_iter = 10 M iterations);
    * the traditional method with the same M cycles per step, one step after another (constant
      b^n per step): N_t M single-column sweeps.
    T_b (forming b, the fused residual) and t_iter (one Arnoldi step) are the single-column
    sweep's split; E1 = N_t / (M + N_t - 1), E2 = (T_b / N_iter + t_iter) / (M / N_iter T_b +
    t_iter). On the GPU the M "threads" are the columns of one multi-RHS sweep, so the measured
    speedup is M E / rho(M), rho(M) the cost of an M-column sweep relative to one column."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2310_10430_gb300 import biot
    case = W.terzaghi_small().with_(n=n, n_t=n_t, precond="diag", name=f"terzaghi_{n}x{n}_nt{n_t}")
    out = {"workload": f"{case.name}: FGMRES(10) cycles, P2, FP64, setup excluded", "rows": []}
    # single-column sweep split: T_b (residual) and t_iter
    with biot.Context(case, stream=stream, window=1) as c:
        biot.biot_tune(c.ctx, None)
        for _ in range(3):
            biot.biot_sweep(c.ctx, 1, 1, want_rel=False)
        torch.cuda.synchronize()
        biot.biot_timing_enable(c.ctx, True)
        reps = 20
        t0 = time.perf_counter()
        for _ in range(reps):
            biot.biot_sweep(c.ctx, 1, 1, want_rel=False)
        torch.cuda.synchronize()
        t1 = (time.perf_counter() - t0) / reps
        res_ms, res_n = biot.biot_timing_read(c.ctx, biot.BIOT_KC_RESIDUAL)
        biot.biot_timing_enable(c.ctx, False)
    T_b = res_ms / res_n / 1e3
    t_iter = max(t1 - T_b, 1e-9) / case.n_iter
    out.update({"T_b_ms": T_b * 1e3, "t_iter_ms": t_iter * 1e3, "sweep_1col_ms": t1 * 1e3})
    for M in Ms:
        with biot.Context(case, stream=stream, window=M, schedule=biot.BIOT_SCHED_PAPER) as c:
            biot.biot_tune(c.ctx, None)
            biot.biot_pint_solve(c.ctx, 0.0, 100000, allow_not_converged=True)  # warm-up
            biot.biot_set_state(c.ctx, 0, case.n_t, np.zeros((case.n_t + 1, case.n_dof)))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, sweeps, rel_p = biot.biot_pint_solve(c.ctx, 0.0, 100000, allow_not_converged=True)
            torch.cuda.synchronize()
            t_pint = time.perf_counter() - t0
        with biot.Context(case, stream=stream, window=1) as c:
            biot.biot_tune(c.ctx, None)
            biot.biot_sweep(c.ctx, 1, 1, want_rel=False)  # warm-up
            biot.biot_set_state(c.ctx, 0, case.n_t, np.zeros((case.n_t + 1, case.n_dof)))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(1, case.n_t + 1):
                for _ in range(M):
                    biot.biot_sweep(c.ctx, k, k, want_rel=False)
            torch.cuda.synchronize()
            t_seq = time.perf_counter() - t0
            rel_s = max(float(biot.biot_residual_norms(c.ctx, k, k)[0]) for k in range(1, case.n_t + 1))
        n_iter_total = case.n_iter * M
        E1 = case.n_t / (M + case.n_t - 1)
        E2 = (T_b / n_iter_total + t_iter) / (M / n_iter_total * T_b + t_iter)
        speedup = t_seq / t_pint
        rho = (t_pint / sweeps) / t1
        out["rows"].append({"N_thread": M, "sweeps": sweeps, "t_pint_s": t_pint, "t_seq_s": t_seq,
                            "speedup": speedup, "E_measured": speedup / M, "E1": E1, "E2": E2, "E1E2": E1 * E2,
                            "rho": rho, "E1E2_over_rho": E1 * E2 / rho,
                            "max_step_residual_pint": float(rel_p), "max_step_residual_seq": rel_s})
    return out


def barry_mercer_study(stream):
    """Barry & Mercer's point source as the paper runs it (Sec. 4.2: 64^2, tau = 1/256, T = 1,
    P2, tol 1e-10): backward Euler one step after another (window 1: each step converged before
    the next) against the parallel-in-time sweep over all 256 steps, in FP64 and with FP32
    sweeps and FP64 refinement; wall times (setup excluded), sweeps, per-field differences."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2310_10430_gb300 import biot
    case = W.barry_mercer()
    out = {"workload": f"{case.name}: P2, tol {case.tol}, setup excluded"}
    ref = None
    for name, window, prec in (("sequential_fp64", 1, "fp64"), ("pint_fp64", 0, "fp64"), ("pint_fp32", 0, "fp32")):
        with biot.Context(case, stream=stream, window=window, precision=prec) as c:
            biot.biot_tune(c.ctx, None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, sweeps, rel = biot.biot_pint_solve(c.ctx, case.tol, 1000000, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            X = biot.biot_get_state(c.ctx, 0, case.n_t)
        row = {"seconds": dt, "sweeps": sweeps, "status": biot.STATUS_NAMES[st], "rel_residual": rel}
        if ref is None:
            ref = X
        else:
            row["rel_diff_u"], row["rel_diff_p"] = _field_errors(np, X, ref)
        out[name] = row
    return out


def mandel_study(stream):
    """Mandel's problem as the paper runs it (Sec. 4.3). (a) The plot's setting: h = 1/32,
    tau = 0.025, P1, tol 1e-7, to t = 10 (400 steps), parallel in time against step by step
    (window 1), FP64; the centre pressure at t = 1, 5, 10 (the Mandel-Cryer rise above the
    undrained 0.5). (b) Near the table's setting: tau = 0.1 on h = 1/64 to T = 20 (200 steps),
    tol 1e-7, P1 against P2, FP32 sweeps with the FP64 refinement."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2310_10430_gb300 import biot
    out = {}
    case = W.mandel(32, 400, 0.025)
    n = case.n
    res = {}
    for label, window in (("pint", 0), ("step_by_step", 1)):
        with biot.Context(case, stream=stream, window=window) as c:
            biot.biot_tune(c.ctx, None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, sweeps, rel = biot.biot_pint_solve(c.ctx, case.tol, 100000, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            X = biot.biot_get_state(c.ctx, 0, case.n_t)
        P = X[:, 2::3].reshape(-1, n + 1, n + 1)
        res[label] = {"seconds": dt, "sweeps": sweeps, "status": biot.STATUS_NAMES[st], "rel_residual": rel,
                      "p_centre": {f"t={k * case.tau:g}": float(P[k, 0, 0]) for k in (40, 200, 400)}}
        res[label]["P"] = P
    # (the comparison with the analytic series is a test: tests/test_gpu_mandel.py)
    diff = float(np.abs(res["pint"]["P"] - res["step_by_step"]["P"]).max() / 0.5)
    for r in res.values():
        r.pop("P")
    out["plot_setting"] = {"workload": "h = 1/32, tau = 0.025, t = 10, P1, tol 1e-7, FP64", **res,
                           "pint_vs_step_by_step_max_dp_over_p0": diff}
    tab = {}
    # the table's tau = 0.1 on h = 1/64 to T = 20 (200 steps): the table's own 128^2 x 1000 steps
    # needs over 1000 sweeps of 1000 columns per solve, more GPU time than a bench extra gets
    case = W.mandel(64, 200, 0.1)
    for kind in ("tri", "diag"):
        with biot.Context(case.with_(precond=kind, n_iter=20), stream=stream, precision="fp32") as c:
            biot.biot_tune(c.ctx, None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, sweeps, rel = biot.biot_pint_solve(c.ctx, case.tol, 20000, allow_not_converged=True)
            torch.cuda.synchronize()
            tab["P1" if kind == "tri" else "P2"] = {"seconds": time.perf_counter() - t0, "sweeps": sweeps,
                                                    "status": biot.STATUS_NAMES[st], "rel_residual": rel}
    out["table_setting"] = {"workload": "h = 1/64, tau = 0.1, T = 20 (200 steps), tol 1e-7, FP32 sweeps with "
                                        "the FP64 refinement, FGMRES(20)", **tab}
    return out


def large_mesh(args, quiet=False):
    """The 1024^2 stress workload (3,151,875 DOF, N_t = 128, nu = 0.49, lognormal kappa sigma 2,
    l = 0.1, P1): FP32 sweeps with the FP64 residual and update. One JSON line: the sweep
    throughput over args.steps timed sweeps (the bench metric, all N_t steps active), the
    setup time (assembly, substructured factorisations) and tuning time, the band-solve
    roofline in FP32, and a tolerance solve to the workload's 1e-8 from the zero state,
    capped at args.large_outer sweeps (0: skipped), with FGMRES(args.large_n_iter)."""
    import torch
    import workloads as W
    from paper_2310_10430_gb300 import biot
    from paper_2310_10430_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    case = W.large_1024()
    if args.large_n_iter:
        case = case.with_(n_iter=args.large_n_iter)
    gmg = GMG if args.large_gmg else None
    ref, ref_run = None, None
    if args.large_outer > 0 and args.large_error and args.large_ref_gmg:
        # the 1e-12 reference from a multigrid context (the faster path), solved and freed before
        # the path under test is set up
        with biot.Context(case.with_(n_iter=max(case.n_iter, 20)), stream=stream, precision="fp32", gmg=GMG) as cr:
            biot.biot_tune(cr.ctx, None)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            st, sweeps, rel = biot.biot_pint_solve(cr.ctx, 1e-12, args.large_outer, allow_not_converged=True)
            torch.cuda.synchronize()
            ref_run = {"seconds": time.perf_counter() - t2, "sweeps": sweeps, "status": biot.STATUS_NAMES[st],
                       "rel_residual": rel, "tol": 1e-12, "block_solves": "multigrid"}
            ref = biot.biot_get_state(cr.ctx, 0, case.n_t)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with biot.Context(case, stream=stream, precision="fp32", strips=args.strips, gmg=gmg) as c:
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        t1 = time.perf_counter()
        tuning = biot.biot_tune(c.ctx, args.tune_cache).as_dict()
        tune_s = time.perf_counter() - t1
        info = c.info
        for _ in range(args.warmup):
            biot.biot_sweep(c.ctx, 1, case.n_t, want_rel=False)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        biot.biot_timing_enable(c.ctx, True)
        l0 = biot.biot_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            biot.biot_sweep(c.ctx, 1, case.n_t, want_rel=False)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = biot.biot_launch_count() - l0
        clk = clocks.stop()
        band_ms, band_n = biot.biot_timing_read(c.ctx, biot.BIOT_KC_BAND_SOLVE)
        biot.biot_timing_enable(c.ctx, False)
        ms = e0.elapsed_time(e1) / args.steps
        rel_swept = float(biot.biot_residual_norms(c.ctx, 1, case.n_t).max())
        solve = None
        time_to_error = None
        if args.large_outer > 0:
            import numpy as np
            zero = np.zeros((case.n_t, case.n_dof))

            def solve_from_zero(tol):
                biot.biot_set_state(c.ctx, 1, case.n_t, zero)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                st, sweeps, rel = biot.biot_pint_solve(c.ctx, tol, args.large_outer, allow_not_converged=True)
                torch.cuda.synchronize()
                return {"seconds": time.perf_counter() - t2, "sweeps": sweeps, "status": biot.STATUS_NAMES[st],
                        "rel_residual": rel, "tol": tol}

            tols = [float(t) for t in args.large_tols.split(",")] if args.large_tols else [case.tol]
            solve = solve_from_zero(tols[0])
            if args.large_error:
                # Error, not residual: at nu = 0.49 the two differ. The reference is the same FP64
                # space-time system solved to a relative FP64 residual of 1e-12 (FP32 sweeps as the
                # correction solver of the FP64 refinement; the path the stress-material tests match
                # against the oracle's backward Euler at 64^2 and 128^2). Each tolerance is solved from
                # the zero state and timed; the time to error 1e-8 is the first whose per-field
                # relative error against the reference is at most 1e-8.
                X = biot.biot_get_state(c.ctx, 0, case.n_t)
                if ref is None:
                    ref_run = solve_from_zero(1e-12)
                    ref = biot.biot_get_state(c.ctx, 0, case.n_t)
                runs = []
                eu, ep = _field_errors(np, X[1:], ref[1:])
                runs.append(dict(solve, err_u=eu, err_p=ep))
                del X
                ladder = tols[1:] if args.large_tols else [1e-9, 1e-10, 1e-11]
                for tol in ladder:
                    if max(runs[-1]["err_u"], runs[-1]["err_p"]) <= 1e-8:
                        break
                    r = solve_from_zero(tol)
                    X = biot.biot_get_state(c.ctx, 0, case.n_t)
                    eu, ep = _field_errors(np, X[1:], ref[1:])
                    runs.append(dict(r, err_u=eu, err_p=ep))
                    del X
                hit = [r for r in runs if max(r["err_u"], r["err_p"]) <= 1e-8]
                time_to_error = {"target": "per-field relative error <= 1e-8 against the 1e-12 reference",
                                 "seconds": hit[0]["seconds"] if hit else None,
                                 "sweeps": hit[0]["sweeps"] if hit else None,
                                 "tol_needed": hit[0]["tol"] if hit else None,
                                 "runs": runs, "reference": ref_run}
                del ref
        device_gb = c.info.device_bytes / 1e9
    hbm, src = _hbm_peak()
    by = sweep_bytes(info, case.n_t, case.n_iter, "fp32", case.precond, int(tuning.get("strips", 0)), gmg=gmg)
    if gmg:
        solves = {"kind": "multigrid V(2,2)-cycles", "levels": info.gmg_levels, "avg_apply_ms": band_ms / band_n,
                  "bytes_per_apply": by["per_apply_block_solves"],
                  "hbm_frac": by["per_apply_block_solves"] / (band_ms / band_n / 1e3) / 1e9 / hbm}
    else:
        fl, per = band_solve_flops(info, case.n_t, case.precond, int(tuning.get("strips", 0)), dense_sep_of(tuning))
        ach = fl / (band_ms / band_n / 1e3) / 1e12
        solves = {"kind": "exact (substructured)", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "bound": "alu", "frac": ach / FP32_PEAK_TFLOPS, "avg_apply_ms": band_ms / band_n,
                  "share_of_step": band_ms / args.steps / ms}
    out = {"metric": METRIC, "value": case.n_dof * case.n_t / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{case.name}: n=1024, N_t=128, nu=0.49, lognormal kappa sigma 2, P1, "
                                  "FP32 sweeps with FP64 residual and update, "
                                  + ("multigrid" if gmg else "exact") + " block solves",
                      "window": case.n_t, "n_iter": case.n_iter, "l2": "inputs larger than L2"},
           "clocks": clk, "gpu_launches": int(launches),
           "setup_seconds": setup_s, "tune_seconds": tune_s, "device_gb": device_gb,
           "block_solves": solves,
           "sweep_roofline": {"bound": "hbm", "algorithmic_bytes": by["total"], "peak": hbm, "peak_source": src,
                              "achieved_gbs": by["total"] / (ms / 1e3) / 1e9,
                              "frac": by["total"] / (ms / 1e3) / 1e9 / hbm},
           "max_rel_residual_after_sweeps": rel_swept, "tolerance_solve": solve,
           "time_to_error": time_to_error, "tuning": tuning}
    if not quiet:
        print(json.dumps(out))
    return out


def batched_vs_sequential(stream, count=16):
    """Config-4-shaped instances (uneven n, N_t, nu, lognormal kappa sigma 1.5), FP32
    with FP64 refinement to 1e-10: one batched solve (CUDA graph) vs the same
    instances solved one after another."""
    import torch
    import workloads as W
    from paper_2310_10430_gb300 import biot
    cases = []
    for inst in W.batched_instances(count):
        n = 32 + 8 * ((inst.n // 8) % 8)   # keep the bench bounded: n in [32, 88]
        nt = 32 + inst.n_t % 64            # N_t in [32, 95]
        cases.append(inst.with_(n=n, n_t=nt, kappa=W.lognormal_kappa(n, sigma=1.5, seed=int(inst.nu * 1e6))))
    ctxs = [biot.Context(c, stream=stream, precision="fp32", precond="tri") for c in cases]
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, sweeps, rels = biot.biot_batch_solve([c.ctx for c in ctxs], 1e-10, 200000, use_graph=True,
                                                 allow_not_converged=True)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
    finally:
        for c in ctxs:
            c.close()
    ctxs = [biot.Context(c, stream=stream, precision="fp32", precond="tri") for c in cases]
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in ctxs:
            biot.biot_pint_solve(c.ctx, 1e-10, 200000, allow_not_converged=True)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
    finally:
        for c in ctxs:
            c.close()
    units = sum(c.n_dof * c.n_t for c in cases)
    return {"instances": count, "n_range": [min(c.n for c in cases), max(c.n for c in cases)],
            "n_t_range": [min(c.n_t for c in cases), max(c.n_t for c in cases)],
            "dof_x_steps": units, "batched_seconds": t_batch, "sequential_seconds": t_seq,
            "speedup": t_seq / t_batch, "max_rel_residual": float(max(rels)), "status": biot.STATUS_NAMES[st]}


def batched_config4(stream, full=False, sweeps=20, count=64):
    """The batched workload at its stated size: 64 instances exactly as
    workloads.batched_instances() draws them (n in [32, 192] multiples of 8, N_t in [64, 512],
    nu in [0.2, 0.45], lognormal kappa sigma 1.5, P1), FP32 sweeps with the FP64 refinement,
    multigrid block solves (every instance keeps its own hierarchy; the batched launches cover
    all of them), FGMRES(10) for the throughput runs and (20) for the tolerance solves.

    Default (bounded GPU time): throughput at equal work -- `sweeps` sweeps with every step of
    every instance active (eager schedule, tol 0), one batched call (CUDA graph) against the
    instances one after another, all 64 instances. full=True: tolerance solves to the FP64
    residual 1e-8 on every 8th instance (8 of the 64; all 64 took more than 40 minutes with the
    plain FP64 comparison), batched and one after another with multigrid FP32 sweeps, and one
    after another with the plain FP64 method (exact block solves, FGMRES(10)); max per-field
    differences between the batched FP32 and the FP64 solutions are reported."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2310_10430_gb300 import biot
    n_iter = 20 if full else 10   # FGMRES(20) converges in fewer sweeps; (10) halves the Krylov memory
    cases = [c.with_(n_iter=n_iter) for c in W.batched_instances(count)]
    units = sum(c.n_dof * c.n_t for c in cases)
    out = {"instances": count, "n_range": [min(c.n for c in cases), max(c.n for c in cases)],
           "n_t_range": [min(c.n_t for c in cases), max(c.n_t for c in cases)], "dof_x_steps": units,
           "block_solves": "multigrid V(2,2)-cycles per instance, batched", "n_iter": n_iter}

    def make(sched, precision="fp32", gmg=GMG, precond=None):
        return [biot.Context(c, stream=stream, precision=precision, schedule=sched, gmg=gmg,
                             precond=precond) for c in cases]

    def close(ctxs):
        for c in ctxs:
            c.close()

    if not full:
        ctxs = make(biot.BIOT_SCHED_EAGER)
        try:
            biot.biot_batch_solve([c.ctx for c in ctxs], 0.0, 2, use_graph=True, allow_not_converged=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            biot.biot_batch_solve([c.ctx for c in ctxs], 0.0, sweeps, use_graph=True, allow_not_converged=True)
            torch.cuda.synchronize()
            t_batch = time.perf_counter() - t0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for c in ctxs:
                biot.biot_pint_solve(c.ctx, 0.0, sweeps, allow_not_converged=True)
            torch.cuda.synchronize()
            t_seq = time.perf_counter() - t0
        finally:
            close(ctxs)
        out.update({"mode": f"{sweeps} sweeps with every step active (eager schedule, tol 0): equal work",
                    "batched_seconds": t_batch, "sequential_seconds": t_seq, "speedup": t_seq / t_batch,
                    "value": units * sweeps / t_batch, "unit": UNIT})
        return out
    res = {}
    cases = cases[::8]
    out.update({"tolerance_instances": [c.name for c in cases], "tolerance_dof_x_steps":
                sum(c.n_dof * c.n_t for c in cases)})
    ctxs = make(biot.BIOT_SCHED_TOL)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, sw, rels = biot.biot_batch_solve([c.ctx for c in ctxs], 1e-8, 200000, use_graph=True,
                                             allow_not_converged=True)
        torch.cuda.synchronize()
        res["batched_fp32_gmg"] = {"seconds": time.perf_counter() - t0, "status": biot.STATUS_NAMES[st],
                                   "max_sweeps": int(max(sw)), "max_rel_residual": float(max(rels))}
        X32 = [biot.biot_get_state(c.ctx, 1, cs.n_t) for c, cs in zip(ctxs, cases)]
    finally:
        close(ctxs)
    ctxs = make(biot.BIOT_SCHED_TOL)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        worst = 0.0
        for c in ctxs:
            st, sw1, rel = biot.biot_pint_solve(c.ctx, 1e-8, 200000, allow_not_converged=True)
            worst = max(worst, rel)
        torch.cuda.synchronize()
        res["sequential_fp32_gmg"] = {"seconds": time.perf_counter() - t0, "max_rel_residual": worst}
    finally:
        close(ctxs)
    diff = 0.0
    t64 = 0.0
    worst = 0.0
    for k, cs in enumerate(cases):
        with biot.Context(cs.with_(n_iter=10), stream=stream) as c:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, sw1, rel = biot.biot_pint_solve(c.ctx, 1e-8, 200000, allow_not_converged=True)
            torch.cuda.synchronize()
            t64 += time.perf_counter() - t0
            worst = max(worst, rel)
            X64 = biot.biot_get_state(c.ctx, 1, cs.n_t)
        diff = max(diff, *_field_errors(np, X32[k], X64))
    res["sequential_fp64_exact"] = {"seconds": t64, "max_rel_residual": worst, "n_iter": 10}
    out.update(res)
    out.update({"mode": "tolerance solves to the FP64 space-time residual 1e-8 from the zero state",
                "speedup_vs_one_after_another": res["sequential_fp32_gmg"]["seconds"] / res["batched_fp32_gmg"]["seconds"],
                "speedup_vs_plain_fp64": t64 / res["batched_fp32_gmg"]["seconds"],
                "max_field_diff_batched_fp32_vs_fp64": diff})
    return out


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return None
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    case = workload()
    n_dof, times = oracle_sample(case, budget_s=1e9, max_cols=args.warmup + args.steps)
    timed = times[args.warmup:]
    ms_per_step = 1e3 * sum(timed) / max(len(timed), 1)
    value = n_dof / (ms_per_step / 1e3)
    sample = (f"each step = one oracle FGMRES({case.n_iter}) cycle with exact sparse-LU block solves on one of "
              f"the {case.n_t} time steps of a full-window sweep at {case.n}x{case.n}")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_dict(case, case.n_t),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-sample", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the reduced-precision, time-to-solution and batched measurements")
    ap.add_argument("--n", type=int, default=None, help="override the mesh size (profiling runs only)")
    ap.add_argument("--nt", type=int, default=None, help="override N_t (profiling runs only)")
    ap.add_argument("--lognormal", type=int, default=0, metavar="N_T",
                    help="also solve the lognormal-permeability 256^2 workload with N_t = N_T in FP64, FP32 "
                         "and BF16 values and report times and errors (off by default: minutes of GPU time)")
    ap.add_argument("--strips", type=int, default=None,
                    help="substructure strip count (profiling runs; default: the library's automatic choice)")
    ap.add_argument("--tune-cache", default=None,
                    help="band-solve tuning cache (JSON): read if present, written otherwise; profiling runs "
                         "use it to replay the plain run's variant choice")
    ap.add_argument("--efficiency", action="store_true",
                    help="also measure the paper's efficiency model (E1, E2) on Terzaghi 64^2, N_t = 64, for "
                         "N_thread = 1 .. 64 (paper schedule against the same cycles step by step)")
    ap.add_argument("--barry-mercer", action="store_true",
                    help="also solve Barry & Mercer's point source (64^2, 256 steps, P2, tol 1e-10) step by "
                         "step and parallel in time, FP64 and FP32, and report times and differences")
    ap.add_argument("--mandel", action="store_true",
                    help="also solve Mandel's problem at the paper's two settings (Sec. 4.3) and report times, "
                         "P1 against P2 and the error against the analytic series")
    ap.add_argument("--batched-full", action="store_true",
                    help="also solve the 64-instance batched workload to 1e-8: batched, one after another and "
                         "with the plain FP64 method (about ten minutes of GPU time)")
    ap.add_argument("--large", action="store_true",
                    help="run only the 1024^2 stress workload (N_t = 128, nu = 0.49, lognormal sigma 2, P1, FP32 "
                         "sweeps with FP64 refinement): setup, --steps timed sweeps, one JSON line")
    ap.add_argument("--large-outer", type=int, default=0,
                    help="with --large: also run the tolerance solve, capped at this many sweeps")
    ap.add_argument("--large-gmg", action="store_true",
                    help="with --large: multigrid block solves instead of the exact substructured ones")
    ap.add_argument("--large-error", action="store_true",
                    help="with --large and --large-outer: also solve to 1e-12 as the reference and time the "
                         "solves until the per-field error (not the residual) is at most 1e-8")
    ap.add_argument("--large-tols", default=None,
                    help="comma-separated tolerance ladder of the --large-error solves (default: the "
                         "workload's 1e-8, then 1e-9, 1e-10, 1e-11 until the error target is met)")
    ap.add_argument("--large-ref-gmg", action="store_true",
                    help="--large-error: solve the 1e-12 reference with multigrid block solves in a "
                         "context of its own (whatever the path under test)")
    ap.add_argument("--large-n-iter", type=int, default=0,
                    help="with --large: FGMRES restart length (default: the workload's 10)")
    ap.add_argument("--gmg", action="store_true",
                    help="multigrid block solves in the timed line (profiling runs; the bench line is exact)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"],
                    help="sweep precision of the timed line (profiling runs; the bench line is fp64)")
    args = ap.parse_args()
    if args.n:
        _SIZE["n"] = args.n
    if args.nt:
        _SIZE["n_t"] = args.nt
    if args.cpu_sample is not None:
        run_cpu_sample(args.cpu_sample)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.large:
        large_mesh(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
