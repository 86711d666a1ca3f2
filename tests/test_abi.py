"""The C-ABI library builds, loads and exports every symbol include/lbm.h declares; host-only
entry points (parameter validation, lattice table, error strings) behave without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_17481_gb300 import binding, build
    build.build()
    return binding


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    L = lib.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_params_struct_matches_header(lib):
    """The ctypes mirror has the header's field order (checked by name)."""
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = txt[txt.index("typedef struct {", txt.index("lbm_store;")):txt.index("} lbm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith("typedef"):
            decl = decl.replace("typedef struct {", "").strip()
            if not decl:
                continue
        decl = re.sub(r"^(int|double)\s+", "", decl)
        for part in decl.split(","):
            fields.append(re.sub(r"\[.*\]", "", part).strip())
    assert fields == [f[0] for f in lib.lbm_params._fields_]


def test_lattice_table_follows_documented_order(lib):
    for dim, Q in ((2, 9), (3, 19), (3, 27)):
        c, w = lib.lbm_lattice(dim, Q)
        keys = [(int(v @ v), int(v[2]), int(v[1]), int(v[0])) for v in c]
        assert keys == sorted(keys)
        assert abs(w.sum() - 1) < 1e-15
        for a in range(3):
            for b in range(3):
                assert abs(np.sum(w * c[:, a] * c[:, b]) - (a == b) * (a < dim) / 3.0) < 1e-15


def test_invalid_parameters_rejected_before_cuda(lib):
    base = lib.lbm_params_default()
    bad = []
    for field, value in [("dim", 4), ("nx", 0), ("Q", 15), ("store", 7), ("rho_g", 0.0), ("nu_l", -1.0),
                         ("eps", 0.0), ("w", 4), ("w", 0), ("q_th", 0.3), ("mass_check_every", -1)]:
        p = lib.lbm_params()
        ctypes.pointer(p)[0] = base
        setattr(p, field, value)
        bad.append((field, p))
    p2 = lib.lbm_params()
    ctypes.pointer(p2)[0] = base
    p2.dim, p2.Q, p2.nz = 2, 9, 4  # 2D needs nz = 1
    bad.append(("nz", p2))
    for field, p in bad:
        with pytest.raises(lib.LbmError) as ei:
            lib.lbm_create(p)
        assert ei.value.code == lib.LBM_ERR_ARG, field


def test_strerror_and_kernel_names(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.lbm_strerror(code)
    assert [lib.lbm_kernel_name(k) for k in range(5)] == list(lib.KERNEL_KINDS)


def test_graft_entry_build_runs():
    import __graft_entry__ as g
    g.build()


def test_lattice_table_equals_the_oracles(lib, orc):
    """The library's velocity sets and weights (compile-time tables) against the oracle's, which
    builds its own from the ordering rule: identical integers and weights."""
    for dim, Q in ((2, 9), (3, 19), (3, 27)):
        c, w = lib.lbm_lattice(dim, Q)
        co, wo = orc.lattice(dim, Q)
        assert np.array_equal(c, co)
        assert np.array_equal(w, wo)


def test_null_handles_rejected_without_a_gpu(lib):
    """Every entry point that takes a context or batch handle rejects a null one before any CUDA call."""
    L = lib.load()
    out = (ctypes.c_double * 8)()
    assert L.lbm_step(None, 1) == lib.LBM_ERR_ARG
    assert L.lbm_mass(None, out, out) == lib.LBM_ERR_ARG
    assert L.lbm_mass_noalloc(None, out, out) == lib.LBM_ERR_ARG
    assert L.lbm_read_fields(None, None, None, None) == lib.LBM_ERR_ARG
    assert L.lbm_nci_diagnostics(None, out) == lib.LBM_ERR_ARG
    assert L.lbm_curvature(None, 0.0, 1.0, 0, None, out) == lib.LBM_ERR_ARG
    assert L.lbm_energy_spectrum(None, 4, out) == lib.LBM_ERR_ARG
    assert L.lbm_batch_step(None, 2) == lib.LBM_ERR_ARG
    assert L.lbm_batch_create(None, 0, 1, None, None) == lib.LBM_ERR_ARG
    assert L.lbm_synchronize(None) == lib.LBM_ERR_ARG
    assert L.lbm_profile(None, 1) == lib.LBM_ERR_ARG
    assert L.lbm_profile_kinds(None, 2) == lib.LBM_ERR_ARG
