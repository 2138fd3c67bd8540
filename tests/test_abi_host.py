"""The C-ABI library loads, exports every declared symbol, and its host-side DoF maps
match the oracle's independent construction bit for bit (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import synthetic as syn
from oracle import mesh as omesh
from paper_2501_18781_gb300 import DofMap, Mesh, _lib, build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_library()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mfgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(mf_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_context_without_gpu_fails_cleanly(lib):
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.mf_context_create(0, None, C.byref(h))
    assert st == _lib.MF_ECUDA and not h.value
    assert b"CUDA" in lib.mf_last_error()


def test_second_device_is_rejected_before_any_cuda_call():
    """The library serves one device per process: after a context request for device 0 (which
    succeeds with a GPU and fails with MF_ECUDA without one), a request for device 1 is refused with
    MF_EUNSUPPORTED, and device 0 is still accepted.  Runs in a fresh process because the binding is
    process-wide."""
    import subprocess
    import sys
    code = (
        "import ctypes as C, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2501_18781_gb300 import _lib\n"
        "lib = _lib.load()\n"
        "h = C.c_void_p()\n"
        "a = lib.mf_context_create(0, None, C.byref(h))\n"
        "if a == 0: lib.mf_context_destroy(h)\n"
        "g = C.c_void_p()\n"
        "b = lib.mf_context_create(1, None, C.byref(g))\n"
        "msg = lib.mf_last_error().decode()\n"
        "c = lib.mf_context_create(0, None, C.byref(h))\n"
        "if c == 0: lib.mf_context_destroy(h)\n"
        "print(a, b, c, 'device 0' in msg and 'one device per process' in msg, bool(g.value))\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    a, b, c, msg_ok, handle = out.stdout.split()
    assert int(a) in (_lib.MF_OK, _lib.MF_ECUDA) and int(c) == int(a)
    assert int(b) == _lib.MF_EUNSUPPORTED and msg_ok == "True" and handle == "False"


def _compare_maps(ours, theirs):
    cm, rp, cols, w = theirs.export()
    e = ours.export()
    assert ours.n_dofs == theirs.n_dofs and ours.n_cells == theirs.n_cells
    assert np.array_equal(e["cell_map"], cm)
    assert np.array_equal(e["con_rowptr"], rp)
    assert np.array_equal(e["con_cols"], cols)
    assert np.array_equal(e["con_w"], w)          # bit-exact dyadic weights
    assert np.array_equal(e["coords"], theirs.dof_coords())
    assert np.array_equal(e["dirichlet"], theirs.dirichlet)


@pytest.mark.parametrize("n,deg,faces", [(1, 2, 0), (3, 2, 0b011111), (4, 1, 0), (5, 2, 0b010000)])
def test_uniform_maps_match_oracle(n, deg, faces):
    lo, hi = (-3e-4,) * 3, (3e-4,) * 3
    ours = DofMap(Mesh.uniform(None, n, lo, hi), deg, faces)
    _compare_maps(ours, omesh.uniform_dofmap(n, lo, hi, deg, faces))


@pytest.mark.parametrize("n,deg", [(1, 3), (3, 3), (2, 4), (3, 4)])
def test_q3_q4_maps_match_oracle(n, deg):
    """Degrees 3 and 4 (Gauss-Lobatto support points): integer maps bit for bit, coordinates to the
    rounding of the closed-form Lobatto points against the oracle's root finder."""
    lo, hi = (-3e-4,) * 3, (3e-4,) * 3
    ours = DofMap(Mesh.uniform(None, n, lo, hi), deg, 0)
    theirs = omesh.uniform_dofmap(n, lo, hi, deg, 0)
    e = ours.export()
    cm, _, _, _ = theirs.export()
    assert ours.n_dofs == theirs.n_dofs and np.array_equal(e["cell_map"], cm)
    assert np.abs(e["coords"] - theirs.dof_coords()).max() <= 1e-15 * 6e-4
    assert not e["dirichlet"].any()


def _leaves_small():
    L = [[0, i, j, k] for k in range(2) for j in range(2) for i in range(2) if (i, j, k) != (0, 0, 0)]
    L += [[1, i, j, k] for k in range(2) for j in range(2) for i in range(2)]
    return np.array(L, dtype=np.int32)


@pytest.mark.parametrize("case", ["corner", "band"])
def test_octree_maps_and_constraints_match_oracle_bit_for_bit(case):
    if case == "corner":
        leaves, base, levels = _leaves_small(), 2, 1
    else:
        d = lambda x, y, z: syn.deformed_sphere_distance(x, y, z, 3)
        leaves, base, levels = syn.refine_band_leaves(4, 2, d, 1.0 / 64), 4, 2
    rng = np.random.default_rng(0)
    shuffled = leaves[rng.permutation(len(leaves))]     # input order must not matter
    ours = DofMap(Mesh.octree(None, base, levels, shuffled), 2, 0)
    theirs = omesh.octree_dofmap(leaves, base, levels)
    assert ours.n_constraints > 0
    _compare_maps(ours, theirs)


def test_octree_rejects_unbalanced_and_bad_tilings():
    from paper_2501_18781_gb300 import MFError
    # a level-2 leaf next to a level-0 leaf across a face
    L = [[0, 1, 0, 0], [0, 0, 1, 0], [0, 1, 1, 0], [0, 0, 0, 1], [0, 1, 0, 1], [0, 0, 1, 1], [0, 1, 1, 1]]
    L += [[1, i, j, k] for k in range(2) for j in range(2) for i in range(2) if (i, j, k) != (1, 1, 1)]
    L += [[2, 2 + i, 2 + j, 2 + k] for k in range(2) for j in range(2) for i in range(2)]
    with pytest.raises(MFError, match="2:1"):
        Mesh.octree(None, 2, 2, np.array(L))
    with pytest.raises(MFError, match="cover"):
        Mesh.octree(None, 2, 1, _leaves_small()[1:])
    with pytest.raises(MFError, match="overlap"):
        Mesh.octree(None, 2, 1, np.concatenate([_leaves_small(), [[0, 0, 0, 0]]]))
    with pytest.raises(MFError, match="cubes"):
        Mesh.uniform(None, (2, 2, 3), (0, 0, 0), (1, 1, 1))
