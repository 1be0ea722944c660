"""Every band-solve variant the tuner can pick gives the same preconditioner.

A cache file naming one variant forces biot_tune to install it; the P^{-1} apply
is then compared with the oracle's exact block solves (FP64: 1e-9, FP32: 1e-3,
per field). A tuning run without a cache picks the fastest feasible variant and
writes the cache.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle.solvers import BlockPreconditioner, field_rel_errors
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()
N_VARIANTS = 7


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("variant", list(range(N_VARIANTS)))
def test_variant_matches_oracle(tmp_path, precision, bound, variant):
    case = W.terzaghi_small().with_(n=20, n_t=5, precond="tri")
    s = build_system(case)
    P = BlockPreconditioner(s, "tri")
    vin = np.random.default_rng(variant).standard_normal((5, s.n_dof))
    with biot.Context(case, precision=precision) as c:
        info = c.info
        tag = "fp64" if precision == "fp64" else "fp32"
        keys = [f"{tag}:N{2 * info.n_nodes}:b{info.band_u}:w{info.window_cap}",
                f"{tag}:N{info.n_nodes}:b{info.band_p}:w{info.window_cap}"]
        path = str(tmp_path / "tune.json")
        with open(path, "w") as f:
            f.write(json.dumps({"band_solve_variants": []})[:-2] + "\n")
            f.write("".join(f'  {{"key": "{k}", "variant": {variant}}},\n' for k in keys) + "]}\n")
        t = biot.biot_tune(c.ctx, path)
        z = biot.biot_precond_apply(c.ctx, vin)
    if t.from_cache:
        assert t.variant_u == variant and t.variant_p == variant
    for k in range(vin.shape[0]):
        ref = P.apply(vin[k])
        eu, ep = field_rel_errors(z[k][None].repeat(2, 0), ref[None].repeat(2, 0))
        assert eu < bound and ep < bound, (variant, eu, ep)


def test_tuning_writes_cache(tmp_path):
    case = W.terzaghi_small().with_(n=24, n_t=8)
    path = str(tmp_path / "tune.json")
    with biot.Context(case) as c:
        t = biot.biot_tune(c.ctx, path)
    assert os.path.exists(path) and t.from_cache == 0
    assert 0 <= t.variant_u < N_VARIANTS and t.ms_u <= t.ms_u_default * 1.05 + 1e-3
    txt = open(path).read()
    assert '"variant"' in txt and json.loads(txt)["band_solve_variants"]


N_SPMM_VARIANTS = 8


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("variant", range(N_SPMM_VARIANTS))
def test_each_spmm_shape_gives_the_same_solution(tmp_path, precision, variant):
    # the SpMM shape (vector width, unrolling, occupancy, grid) changes only the order of the
    # norm partials: the converged FP32 + refinement solve must still reach backward Euler
    from oracle.solvers import seq_solve
    case = W.terzaghi_small().with_(n=20, n_t=12, precond="tri")
    ref = seq_solve(build_system(case))
    with biot.Context(case, precision=precision) as c:
        key = f"spmm:{precision}:N{case.n_dof}:w{c.info.window_cap}"
        forced = tmp_path / "spmm.json"
        forced.write_text('{"band_solve_variants": [\n' + f'  {{"key": "{key}", "variant": {variant}}}\n' + "]}\n")
        t = biot.biot_tune(c.ctx, str(forced))
        assert t.spmm_variant == variant
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 20000, allow_not_converged=(precision == "bf16"))
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    if rel <= 1e-12:
        eu, ep = field_rel_errors(X, ref)
        assert eu < 1e-8 and ep < 1e-8, (variant, eu, ep)


def test_spmm_tuner_picks_and_caches(tmp_path):
    case = W.terzaghi_small().with_(n=48, n_t=64)
    cache = tmp_path / "tune.json"
    with biot.Context(case, precision="fp32") as c:
        t = biot.biot_tune(c.ctx, str(cache))
        assert 0 <= t.spmm_variant < N_SPMM_VARIANTS and t.ms_spmm <= t.ms_spmm_default * 1.0001
        entries = json.loads(cache.read_text())["band_solve_variants"]
        assert any(e["key"].startswith("spmm:fp32:") for e in entries)
        t2 = biot.biot_tune(c.ctx, str(cache))
        assert t2.spmm_variant == t.spmm_variant and t2.from_cache == 1


def test_cached_default_spmm_shape_hits_on_a_ragged_window(tmp_path):
    # a window that is not a multiple of four columns: the vector shapes do not fit, and a cached
    # default shape (the scalar kernel there) must still count as a cache hit
    case = W.terzaghi_small().with_(n=16, n_t=6)
    with biot.Context(case, precision="fp32") as c:
        assert c.info.window_cap % 4 != 0
        cache = tmp_path / "tune.json"
        biot.biot_tune(c.ctx, str(cache))
        entries = json.loads(cache.read_text())["band_solve_variants"]
        for e in entries:
            if e["key"].startswith("spmm:"):
                e["variant"] = 0
        cache.write_text('{"band_solve_variants": [\n' +
                         ",\n".join(f'  {{"key": "{e["key"]}", "variant": {e["variant"]}}}' for e in entries) + "\n]}\n")
        t = biot.biot_tune(c.ctx, str(cache))
        assert t.spmm_variant == 0 and t.from_cache == 1
