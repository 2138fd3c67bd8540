"""mf_autotune's cache: a record keyed by the operator's configuration is appended after timing,
and a later call with the same cache file applies the stored choice instead of timing again."""
import json

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def _heat(ctx, n=6):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    wl = syn.scaled(syn.HEAT_LASER, n)
    p = wl.params
    m = DofMap(Mesh.uniform(ctx, n, wl.lo, wl.hi), 2, 1 << 4)
    T = torch.tensor(syn.heat_initial_temperature(*m.coords().T, p["laser"]["radius"], wl.hi[2]), device="cuda")
    op = Operator(ctx, "heat", [m], rhocp=p["rhocp"], dt=p["dt"], k0=p["k0"], t_boil=p["t_boil"])
    op.set_field("t_prev", T)
    op._keep = T
    return op, m


def _f32_variant(op, n):
    u = torch.tensor(syn.uniform_pm1(1, n), device="cuda").float()
    op.apply(u)
    return op.variant


def test_autotune_cache_is_written_then_read_back(ctx, tmp_path):
    path = str(tmp_path / "tune.jsonl")
    op, m = _heat(ctx)
    op.autotune(path)
    lines = open(path).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert "key" in rec and "timings" in rec and rec["mode32"] in (0, 1)
    # the same configuration again: the stored choice is applied, nothing is appended
    op2, _ = _heat(ctx)
    op2.autotune(path)
    assert len(open(path).read().splitlines()) == 1
    assert _f32_variant(op2, m.n_dofs) == _f32_variant(op, m.n_dofs)
    # a record that forces the other fp32 coefficient mode is honoured (the last matching record wins);
    # it also selects one thread per cell, the kernel whose variant shows the coefficient mode
    forced = dict(rec, mode32=1 - rec["mode32"], q2_line32=0)
    with open(path, "a") as f:
        f.write(json.dumps(forced) + "\n")
    op3, _ = _heat(ctx)
    op3.autotune(path)
    want = "/tabulated" if forced["mode32"] == 1 else "/inkernel"
    assert want in _f32_variant(op3, m.n_dofs)
    # so is the choice of one or nine threads per cell (the line-per-thread kernel)
    assert rec["q2_line32"] in (0, 1) and rec["q2_line64"] in (0, 1)
    line = dict(rec, q2_line32=1 - rec["q2_line32"])
    with open(path, "a") as f:
        f.write(json.dumps(line) + "\n")
    op5, _ = _heat(ctx)
    op5.autotune(path)
    assert ("line-per-thread" in _f32_variant(op5, m.n_dofs)) == bool(line["q2_line32"])
    # another configuration (other mesh size) does not match the key: it is timed and appended
    op4, _ = _heat(ctx, 5)
    op4.autotune(path)
    assert len(open(path).read().splitlines()) == 4
