"""Substructured exact block solves (strips + separator Schur complement) against the oracle.

The preconditioner's blocks A and S are solved exactly either by plain band Cholesky in
natural order or, with biot_set_substructure(k), by k strips whose interiors are factored
along their short side plus the factored Schur complement of the k - 1 separator lines.
Both are exact, so a P^{-1} apply must match the oracle's sparse-LU block solves to within
cond(block) * eps (1e-9 relative per field in FP64, 1e-3 with the FP32-rounded factors),
and a converged PinT solve must match backward Euler to the FP64 parity bound 1e-10.
The strip counts cover uneven strip widths, the narrowest legal strips (two node columns)
and ragged windows; the automatic choice (about 18 node columns per strip in FP64) is checked at n = 64.
"""
import json

import numpy as np
import pytest

import workloads as W
from oracle.solvers import BlockPreconditioner, field_rel_errors, seq_solve
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


def apply_errors(case, kind, strips, precision, ncols=4, seed=5):
    s = build_system(case)
    P = BlockPreconditioner(s, kind)
    vin = np.random.default_rng(seed).standard_normal((ncols, s.n_dof))
    with biot.Context(case, precision=precision, precond=kind, strips=strips) as c:
        t = biot.biot_tune(c.ctx, None)
        z = biot.biot_precond_apply(c.ctx, vin)
    worst = 0.0
    for k in range(ncols):
        ref = P.apply(vin[k])
        eu, ep = field_rel_errors(z[k][None].repeat(2, 0), ref[None].repeat(2, 0))
        worst = max(worst, eu, ep)
    return worst, t


@pytest.mark.parametrize("kind", ["diag", "tri"])
@pytest.mark.parametrize("n,strips", [(16, 2), (20, 3), (24, 4), (22, 8)])
def test_apply_matches_oracle_fp64(kind, n, strips):
    case = W.terzaghi_small().with_(n=n, n_t=6)
    err, t = apply_errors(case, kind, strips, "fp64")
    assert t.strips == strips
    assert err < 1e-9, err


@pytest.mark.parametrize("kind", ["diag", "tri"])
def test_apply_matches_oracle_fp32(kind):
    case = W.terzaghi_small().with_(n=20, n_t=5)
    err, t = apply_errors(case, kind, 3, "fp32")
    assert t.strips == 3
    assert err < 1e-3, err


def test_apply_lognormal_and_mms():
    base = W.terzaghi_small()
    for case in (base.with_(n=18, kappa=W.lognormal_kappa(18, sigma=1.5, seed=3), nu=0.45, n_t=3),
                 base.with_(n=17, problem="mms", E=3.0, nu=0.25, kappa=0.7, tau=0.05, n_t=3)):
        err, _ = apply_errors(case, "tri", 3, "fp64", ncols=3)
        assert err < 1e-9, err


def test_substructured_equals_plain_band():
    case = W.terzaghi_small().with_(n=24, n_t=8)
    vin = np.random.default_rng(9).standard_normal((8, case.n_dof))
    out = []
    for strips in (1, 5):
        with biot.Context(case, strips=strips) as c:
            out.append(biot.biot_precond_apply(c.ctx, vin))
    eu, ep = field_rel_errors(out[1], out[0])
    assert eu < 1e-10 and ep < 1e-10, (eu, ep)


def test_automatic_strips_at_n64():
    case = W.terzaghi_small().with_(n=64, n_t=3)
    err, t = apply_errors(case, "diag", None, "fp64", ncols=3)
    assert t.strips == 4  # about 18 node columns per strip in FP64
    assert err < 1e-9, err


@pytest.mark.parametrize("kind", ["diag", "tri"])
def test_converged_solve_matches_sequential(kind):
    case = W.terzaghi_small().with_(precond=kind, n_t=12)
    s = build_system(case)
    Xs = seq_solve(s)
    with biot.Context(case, strips=3, window=5) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-13, 100000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, Xs)
    assert st == biot.BIOT_OK and eu < 1e-10 and ep < 1e-10, (eu, ep)
    assert rel < 1e-12


def test_mixed_precision_solve_with_strips():
    case = W.terzaghi_small().with_(n=20, n_t=8)
    s = build_system(case)
    Xs = seq_solve(s)
    with biot.Context(case, strips=3, precision="fp32") as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 100000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, Xs)
    assert st == biot.BIOT_OK and eu < 1e-8 and ep < 1e-8, (eu, ep)


def test_invalid_strip_counts():
    ctx = biot.biot_mesh_create(10)
    try:
        for bad in (-1, 5, 100):  # 3 k > n + 2 leaves fewer than two columns per strip
            with pytest.raises(biot.BiotError) as e:
                biot.biot_set_substructure(ctx, bad)
            assert e.value.status == biot.BIOT_E_INVALID
        for ok in (0, 1, 2, 4):
            biot.biot_set_substructure(ctx, ok)
    finally:
        biot.biot_destroy(ctx)


def test_bf16_values_with_strips_and_narrow_window():
    case = W.terzaghi_small().with_(n=20, n_t=10)
    s = build_system(case)
    Xs = seq_solve(s)
    for precision, window in (("bf16", 0), ("fp32", 3)):
        with biot.Context(case, strips=4, precision=precision, window=window) as c:
            st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 100000)
            X = biot.biot_get_state(c.ctx, 0, case.n_t)
        eu, ep = field_rel_errors(X, Xs)
        assert st == biot.BIOT_OK and eu < 1e-8 and ep < 1e-8, (precision, window, eu, ep)


def test_resetup_switches_between_plain_and_strips():
    # a second biot_precond_setup rebuilds (or drops) the substructure and frees the old one
    case = W.terzaghi_small().with_(n=20, n_t=4)
    s = build_system(case)
    vin = np.random.default_rng(2).standard_normal((4, s.n_dof))
    with biot.Context(case, strips=3) as c:
        bytes0 = c.info.device_bytes
        outs = []
        for strips, kind in ((1, "tri"), (4, "diag"), (3, "tri")):
            biot.biot_set_substructure(c.ctx, strips)
            biot.biot_precond_setup(c.ctx, biot._PRECOND[kind])
            z = biot.biot_precond_apply(c.ctx, vin)
            P = BlockPreconditioner(s, kind)
            err = max(max(field_rel_errors(z[k][None].repeat(2, 0), P.apply(vin[k])[None].repeat(2, 0)))
                      for k in range(4))
            assert err < 1e-9, (strips, kind, err)
            outs.append(c.info.device_bytes)
        assert outs[-1] <= bytes0 * 1.01, (bytes0, outs)  # no growth after returning to 3 strips


WIDE_VARIANT = 10  # four-row TMA blocks: the separator solve of large meshes
DENSE_SEP = 100    # separators by dense block products with the inverted diagonal blocks


def forced_apply(tmp_path, case, precision, variant, separators, seed, strips=4):
    """P^{-1} apply with the interior (or separator) solves forced to one variant.

    A tuning cache naming a variant forces it. Keys are "sub:<precision>:N<rows>:b<half-band>:w<window>"."""
    s = build_system(case)
    vin = np.random.default_rng(seed).standard_normal((5, s.n_dof))
    with biot.Context(case, precision=precision, strips=strips) as c:
        probe = tmp_path / "probe.json"
        biot.biot_tune(c.ctx, str(probe))
        entries = json.loads(probe.read_text())["band_solve_variants"]
        for e in entries:
            if not e["key"].startswith("sub:"):
                continue  # the SpMM shape of the reduced-precision sweep ("spmm:...") keeps its choice
            # separators have half-band 2 d (n + 1) - 1 (d = 1, 2), strip interiors d (w + 2) - 1
            if (int(e["key"].split(":b")[1].split(":")[0]) >= 2 * (case.n + 1) - 1) == separators:
                e["variant"] = variant
        forced = tmp_path / "forced.json"  # the library reads one entry per line
        forced.write_text('{"band_solve_variants": [\n' +
                          "".join(f'  {{"key": "{e["key"]}", "variant": {e["variant"]}}},\n' for e in entries) + "]}\n")
        t = biot.biot_tune(c.ctx, str(forced))
        z = biot.biot_precond_apply(c.ctx, vin)
    assert t.from_cache == 1
    P = BlockPreconditioner(s, case.precond)
    worst = 0.0
    for k in range(vin.shape[0]):
        worst = max(worst, *field_rel_errors(z[k][None].repeat(2, 0), P.apply(vin[k])[None].repeat(2, 0)))
    return t, worst


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("variant", [1, 2, 3, 5, 7, 8, 9, WIDE_VARIANT])
def test_each_interior_variant(tmp_path, precision, bound, variant):
    # separators keep the tuned choice
    case = W.terzaghi_small().with_(n=22, n_t=6)
    t, err = forced_apply(tmp_path, case, precision, variant, separators=False, seed=variant)
    assert t.variant_u == variant and t.variant_p == variant
    assert err < bound, (variant, err)


@pytest.mark.parametrize("kind", ["diag", "tri"])
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("variant", [1, 4, 5, WIDE_VARIANT, DENSE_SEP])
def test_each_separator_variant(tmp_path, kind, precision, bound, variant):
    # band substitutions (with the block-bidiagonal skip; four-row blocks for large meshes) and
    # the dense block products, on a ragged set of columns (5: two column pairs and a lone one)
    case = W.terzaghi_small().with_(n=23, n_t=7, precond=kind)
    t, err = forced_apply(tmp_path, case, precision, variant, separators=True, seed=11)
    assert t.variant_sep_u == variant and t.variant_sep_p == variant
    assert err < bound, (variant, err)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("strips", [2, 3, 6])
def test_dense_separators_chain_lengths(tmp_path, precision, bound, strips):
    # one separator block (no chain products), two (one per direction) and five
    case = W.terzaghi_small().with_(n=21, n_t=5, precond="tri")
    t, err = forced_apply(tmp_path, case, precision, DENSE_SEP, separators=True, seed=strips, strips=strips)
    assert t.strips == strips and t.variant_sep_u == DENSE_SEP
    assert err < bound, (strips, err)


def test_large_mesh_without_natural_order_factors(tmp_path):
    # Above n = 512 a substructured context builds no natural-order band factors (A's alone
    # would hold 8.9 GB at n = 520). Its separators (blocks of 2 * 521 rows, half-band
    # 4 * 521 - 1 = 2083) are solved both ways: by the dense block products and by the band
    # substitution in four-row blocks (the only staging that fits). A property that holds at
    # any size checks the solves: P2 inverts the assembled blocks, A z_u = r_u and
    # AA_pp z_p = r_p, checked on the host with the library's CSR (whose pattern and values
    # match the oracle's at small sizes).
    sp = pytest.importorskip("scipy.sparse")
    case = W.terzaghi_small().with_(n=520, n_t=3, precond="diag")
    vin = np.random.default_rng(4).standard_normal((3, case.n_dof))
    zs = []
    with biot.Context(case) as c:
        probe = tmp_path / "probe.json"
        t = biot.biot_tune(c.ctx, str(probe))
        assert t.strips == 20  # min((n + 10) / 18, sqrt((n + 1) / 1.31)) in FP64
        for variant in (DENSE_SEP, WIDE_VARIANT):
            entries = json.loads(probe.read_text())["band_solve_variants"]
            forced = tmp_path / f"forced{variant}.json"
            forced.write_text('{"band_solve_variants": [\n' + "".join(
                f'  {{"key": "{e["key"]}", "variant": '
                f'{variant if int(e["key"].split(":b")[1].split(":")[0]) >= 2 * (case.n + 1) - 1 else e["variant"]}}},\n'
                for e in entries) + "]}\n")
            t = biot.biot_tune(c.ctx, str(forced))
            assert t.from_cache == 1 and t.variant_sep_u == variant and t.variant_sep_p == variant
            zs.append(biot.biot_precond_apply(c.ctx, vin))
        rowptr, col, val, _ = biot.biot_get_csr(c.ctx)
        with pytest.raises(biot.BiotError) as e:
            biot.biot_batch_solve([c.ctx], 1e-8, 10)
        assert e.value.status == biot.BIOT_E_INVALID
    K = sp.csr_matrix((val, col, rowptr), shape=(len(rowptr) - 1,) * 2)
    nd = K.shape[0]
    u = np.flatnonzero(np.arange(nd) % 3 != 2)
    p = np.arange(2, nd, 3)
    Auu, App = K[u][:, u], K[p][:, p]
    for z in zs:
        for k in range(vin.shape[0]):
            ru = np.linalg.norm(Auu @ z[k, u] - vin[k, u]) / np.linalg.norm(vin[k, u])
            rp = np.linalg.norm(App @ z[k, p] - vin[k, p]) / np.linalg.norm(vin[k, p])
            assert ru < 1e-10 and rp < 1e-10, (k, ru, rp)
