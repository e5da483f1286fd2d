"""Host-side checks of the C ABI (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ahlp.h")


def _lib():
    from paper_2412_07731_gb300 import _lib as L
    if not os.path.exists(L.lib_path()):
        import __graft_entry__
        __graft_entry__.build()
    return L


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?!typedef)(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("arrowhead_lp_create", "ipm_solve", "kkt_factor", "kkt_solve",
               "kkt_adjoint_solve"):
        assert fn in names


def test_library_exports_every_declared_symbol():
    L = _lib()
    lib = ctypes.CDLL(L.lib_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(L.EXPORTS)


def test_default_options_and_status_strings():
    L = _lib()
    o = L.default_options()
    assert o.precision == 0 and o.max_iter == 200
    assert o.tol == 1e-8 and o.refine_tol == 1e-10 and o.eta == 0.9995
    assert o.ipm_refine_tol == 1e-6 and o.fp32_cond_max == 1e14
    lib = L.load()
    assert lib.ahlp_status_string(-4) == b"NOT_SPD"
    assert lib.ahlp_status_string(0) == b"OK"


def _small_lp():
    from instances import config0
    return config0()


def _create_status(lp, batch=1, options=None):
    L = _lib()
    lib = L.load()
    keep = L._Keep()
    lps = lp if isinstance(lp, list) else [lp] * max(batch, 1)
    descs = (L.Desc * max(batch, 1))()
    for k in range(max(batch, 1)):
        descs[k] = L.make_desc(lps[k], keep)
    h = ctypes.c_void_p()
    st = lib.arrowhead_lp_create(descs, batch, ctypes.byref(options) if options else None,
                                 ctypes.byref(h))
    if st == 0:
        lib.arrowhead_lp_destroy(h)
    return st, lib.ahlp_last_error(None).decode()


def test_validation_nan_rhs():
    lp = _small_lp()
    lp.b[1] = lp.b[1].copy()
    lp.b[1][3] = np.nan
    st, msg = _create_status(lp)
    assert st == -1 and "non-finite" in msg


def test_validation_bad_shape():
    lp = _small_lp()
    lp.W[2] = sp.csc_matrix(np.ones((lp.A[2].shape[0], lp.n0 + 1)))
    st, msg = _create_status(lp)
    assert st == -2 and "W" in msg


def test_validation_row_index_out_of_range():
    lp = _small_lp()
    A = lp.A[0].copy()
    A.indices = A.indices.copy()
    A.indices[0] = A.shape[0] + 5
    lp.A[0] = A
    st, msg = _create_status(lp)
    assert st == -1 and "out of range" in msg


def test_batch_validation_and_bad_precision():
    lp = _small_lp()
    st, msg = _create_status(lp, batch=0)
    assert st == -1 and "batch" in msg
    bad = _small_lp()
    bad.W[1] = sp.csc_matrix(np.ones((bad.A[1].shape[0], bad.n0 + 1)))
    st, msg = _create_status([lp, bad], batch=2)   # composing the batch checks shapes
    assert st == -2 and "batch" in msg
    L = _lib()
    st, msg = _create_status(lp, options=L.default_options(precision=7))
    assert st == -1 and "precision" in msg
    st, msg = _create_status(lp, options=L.default_options(ipm_refine_tol=1.5))
    assert st == -1 and "option" in msg


def test_valid_problem_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, msg = _create_status(_small_lp())
    assert st == -8
    st, msg = _create_status(_small_lp(), batch=3)   # a valid batch also gets that far
    assert st == -8


def test_ctypes_structures_match_the_header(tmp_path):
    """The binding's ctypes mirrors of the C structs have the header's sizes
    and field offsets (a C program compiled against include/ahlp.h prints
    them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    L = _lib()
    pairs = [("ahlp_csc", L.CSC), ("ahlp_desc", L.Desc), ("ahlp_options", L.Options),
             ("ahlp_result", L.Result), ("ahlp_solve_info", L.SolveInfo)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ahlp.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in pairs:
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_validation_reports_the_first_failing_block():
    """Blocks are validated concurrently; the error is still the one of the
    lowest-numbered bad block, whatever the thread timing."""
    from instances import random_block_lp
    lp = random_block_lp(2, N=12, m_sizes=[30] * 12, n_sizes=[45] * 12, nnz_per_col=3, n0=2,
                         w_density=0.3, l=[2] * 11, mg=1, global_nnz=3)
    lp.A[3] = lp.A[3].copy()
    lp.A[3].data[0] = np.nan
    lp.A[9] = lp.A[9].copy()
    lp.A[9].data[0] = np.inf
    for _ in range(5):
        st, msg = _create_status(lp)
        assert st == -1 and "block 3" in msg and "non-finite" in msg, msg


def _general_status(mutate):
    from instances import general_block_lp
    lp = general_block_lp(3, N=3, m=12, n=18)
    mutate(lp)
    return _create_status(lp)


def test_full_statement_validation():
    """The full statement is checked and reduced on the host before any device
    work: inconsistent bounds and inequality rows are rejected by name, and a
    valid LP in the full statement gets as far as the device (no GPU here)."""
    torch = pytest.importorskip("torch")

    def lo_above_hi(lp):
        lp.lb[1] = lp.lb[1].copy()
        lp.ub[1] = lp.ub[1].copy()
        lp.lb[1][2], lp.ub[1][2] = 1.0, 0.5

    def nan_bound(lp):
        lp.ub0 = lp.ub0.copy()
        lp.ub0[0] = np.nan

    def row_lo_above_hi(lp):
        lp.dlo[0] = lp.dlo[0].copy()
        lp.dhi[0] = lp.dhi[0].copy()
        lp.dlo[0][1], lp.dhi[0][1] = 2.0, -2.0

    def infinite_lower_row(lp):
        lp.gglo = np.full_like(lp.gglo, np.inf)

    def nan_in_D(lp):
        lp.D[2] = lp.D[2].copy()
        lp.D[2].data[0] = np.nan

    for mutate, words in ((lo_above_hi, "bounds"), (nan_bound, "bounds"),
                          (row_lo_above_hi, "bounds"), (infinite_lower_row, "bounds"),
                          (nan_in_D, "NaN")):
        st, msg = _general_status(mutate)
        assert st == -1 and words in msg, (mutate.__name__, st, msg)
    if not torch.cuda.is_available():
        st, msg = _general_status(lambda lp: None)
        assert st == -8, msg


@pytest.mark.parametrize("bad", [dict(tile_sparse=2), dict(tile_sparse=-1), dict(pivot_mode=2),
                                 dict(fp32_update=4), dict(ff_update=-1), dict(schur_chain=2),
                                 dict(max_correctors=9), dict(eta=1.0), dict(tol=0.0),
                                 dict(fp32_cond_max=0.5), dict(profile_kernels=3),
                                 dict(correctors_by_cost=2)])
def test_option_ranges_are_checked(bad):
    L = _lib()
    st, msg = _create_status(_small_lp(), options=L.default_options(**bad))
    assert st == -1 and "option" in msg, (bad, st, msg)
