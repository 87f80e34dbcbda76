"""The C-ABI library: loads, exports every function include/pcdn.h declares, rejects bad input on
the host (no GPU needed for any of these)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pk():
    from paper_1306_4080_gb300 import build
    build.build()
    import paper_1306_4080_gb300 as m
    m.load()
    return m


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pcdn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pcdn_[A-Za-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(pk):
    names = declared_functions()
    assert len(names) >= 13
    out = subprocess.run(["nm", "-D", "--defined-only", pk.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pcdn_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(pk.LIB_PATH)
    for n in names:
        assert hasattr(lib, n)
    assert sorted(pk.SYMBOLS) == names


def test_default_opts(pk):
    o = pk.pcdn_default_opts()
    assert (o.sigma, o.beta, o.gamma, o.nu) == (0.01, 0.5, 0.0, 1e-12)
    assert o.q_max == 30 and o.max_epochs == 1000 and o.prec == 0 and o.refresh == 1


def _good():
    col_ptr = np.array([0, 2, 3, 3, 5], dtype=np.int64)
    row_idx = np.array([0, 2, 1, 0, 2], dtype=np.int32)
    val = np.array([1.0, 0.5, -2.0, 0.25, 1.0], dtype=np.float32)
    y = np.array([1, -1, 1], dtype=np.int8)
    return col_ptr, row_idx, val, y


@pytest.mark.parametrize("case", ["col_ptr_start", "col_ptr_decreasing", "row_out_of_range", "rows_not_ascending",
                                  "nan_value", "bad_label", "bad_C", "bad_loss"])
def test_create_rejects_bad_input_on_host(pk, case):
    col_ptr, row_idx, val, y = _good()
    C, loss = 1.0, "logistic"
    if case == "col_ptr_start":
        col_ptr = col_ptr.copy(); col_ptr[0] = 1
    elif case == "col_ptr_decreasing":
        col_ptr = np.array([0, 3, 2, 3, 5], dtype=np.int64)
    elif case == "row_out_of_range":
        row_idx = row_idx.copy(); row_idx[1] = 3
    elif case == "rows_not_ascending":
        row_idx = np.array([2, 0, 1, 0, 2], dtype=np.int32)
    elif case == "nan_value":
        val = val.copy(); val[2] = np.nan
    elif case == "bad_label":
        y = np.array([1, 0, 1], dtype=np.int8)
    elif case == "bad_C":
        C = 0.0
    elif case == "bad_loss":
        loss = None
    if case == "bad_loss":
        lib = pk.load()
        X = pk.pcdn_csc(3, 4, 5, col_ptr.ctypes.data, row_idx.ctypes.data, val.ctypes.data)
        h = ctypes.c_void_p()
        rc = lib.pcdn_create(ctypes.byref(X), y.ctypes.data, 1.0, 7, ctypes.byref(h))
        assert rc == pk.PCDN_EINVAL and h.value is None
        return
    with pytest.raises(pk.PcdnError) as ei:
        pk.pcdn_create(col_ptr, row_idx, val, y, C, loss)
    assert ei.value.code == pk.PCDN_EINVAL
    assert pk.pcdn_last_error()


def test_null_arguments_are_errors(pk):
    lib = pk.load()
    assert lib.pcdn_solve(None, 1, 1e-3, 0, None, None, None, None) == pk.PCDN_EINVAL
    assert lib.pcdn_set_w(None, None) == pk.PCDN_EINVAL
    lib.pcdn_destroy(None)


def test_no_device_is_reported(pk, has_cuda):
    if has_cuda:
        pytest.skip("a CUDA device is present")
    col_ptr, row_idx, val, y = _good()
    with pytest.raises(pk.PcdnError) as ei:
        pk.pcdn_create(col_ptr, row_idx, val, y, 1.0, "logistic")
    assert ei.value.code == pk.PCDN_ECUDA


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1306_4080_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "pcdn_oracle" not in txt, f


def test_batch_and_server_validate_on_host(pk, has_cuda):
    lib = pk.load()
    bs = pk.pcdn_batch_stats()
    # an empty batch is a no-op; a job without a problem or C path is rejected before any device work
    assert lib.pcdn_solve_batch(None, 0, None, None, ctypes.byref(bs)) == pk.PCDN_OK
    assert bs.solves == 0
    jobs = (pk.pcdn_batch_job * 1)()
    assert lib.pcdn_solve_batch(jobs, 1, None, None, None) == pk.PCDN_EINVAL
    assert "problem" in pk.pcdn_last_error()
    assert lib.pcdn_solve_batch(None, -1, None, None, None) == pk.PCDN_EINVAL
    bo = pk.pcdn_default_batch_opts()
    assert bo.probe_eps == 0.1 and bo.probe_epochs == 3 and bo.max_inflight == 0
    Pb = ctypes.c_int32()
    assert lib.pcdn_autotune(None, None, 0, 0.1, 3, 0, None, ctypes.byref(Pb), None) == pk.PCDN_EINVAL
    assert lib.pcdn_set_C(None, 1.0) == pk.PCDN_EINVAL
    so = pk.pcdn_server_opts()
    lib.pcdn_default_server_opts(ctypes.byref(so))
    assert so.hbm_budget == 8 << 30 and so.slots == 0 and so.solve.q_max == 30
    so.slots = -1
    h = ctypes.c_void_p()
    assert lib.pcdn_server_create(ctypes.byref(so), ctypes.byref(h)) == pk.PCDN_EINVAL
    assert lib.pcdn_server_submit(None, None, None, 1.0, 0, 1, 1e-3, 0, None) == pk.PCDN_EINVAL
    assert lib.pcdn_server_wait(None, 1, 0.0, None, None) == pk.PCDN_EINVAL
    assert lib.pcdn_server_stats(None, None, None, None, None) == pk.PCDN_EINVAL
    lib.pcdn_server_destroy(None)
    if not has_cuda:
        lib.pcdn_default_server_opts(ctypes.byref(so))
        assert lib.pcdn_server_create(ctypes.byref(so), ctypes.byref(h)) == pk.PCDN_ECUDA


def test_host_validation_of_a_large_csc_reports_the_first_bad_column(pk):
    # above 2^20 nonzeros the host check runs on several threads over column ranges; the message
    # must still name the lowest failing column
    rng = np.random.default_rng(0)
    n, m, per = 4096, 20000, 64
    cols = [np.unique(r) for r in rng.integers(0, n, size=(m, per))]  # ascending rows per column
    col_ptr = np.zeros(m + 1, dtype=np.int64)
    col_ptr[1:] = np.cumsum([len(c) for c in cols])
    ri = np.concatenate(cols).astype(np.int32)
    assert ri.shape[0] >= (1 << 20)
    val = np.ones(ri.shape[0], dtype=np.float32)
    y = np.ones(n, dtype=np.int8)
    bad_late, bad_early = 17000, 9001
    v2 = val.copy()
    v2[col_ptr[bad_late] + 1] = np.inf
    r2 = ri.copy()
    a = col_ptr[bad_early]
    r2[a], r2[a + 1] = r2[a + 1], r2[a]
    with pytest.raises(pk.PcdnError) as ei:
        pk.pcdn_create(col_ptr, r2, v2, y, 1.0, "logistic")
    assert ei.value.code == pk.PCDN_EINVAL and f"column {bad_early}" in str(ei.value)
    with pytest.raises(pk.PcdnError) as ei:
        pk.pcdn_create(col_ptr, ri, v2, y, 1.0, "logistic")
    assert ei.value.code == pk.PCDN_EINVAL and f"column {bad_late}" in str(ei.value)
    cp = col_ptr.copy()
    cp[5000] = 10**12  # a column pointer beyond nnz is caught before any entry is read
    with pytest.raises(pk.PcdnError) as ei:
        pk.pcdn_create(cp, ri, val, y, 1.0, "logistic")
    assert ei.value.code == pk.PCDN_EINVAL and "column 4999" in str(ei.value)


STRUCTS = ["pcdn_csc", "pcdn_opts", "pcdn_stats", "pcdn_trace", "pcdn_batch_job", "pcdn_batch_opts",
           "pcdn_batch_stats", "pcdn_server_opts", "pcdn_request_info"]


def test_binding_structs_match_the_header_layout(pk, tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (a C program built
    against include/pcdn.h prints them)."""
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pcdn.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(pk, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name in STRUCTS:
        cls = getattr(pk, name)
        assert c_layout[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert c_layout[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_penalty_rejects_a_missing_problem(pk):
    """pcdn_set_penalty validates on the host (no GPU needed for the error path)."""
    lib = pk.load()
    assert lib.pcdn_set_penalty(None, 1.0, 0.0) == pk.PCDN_EINVAL
    assert "problem" in pk.pcdn_last_error()


def test_every_declaration_cites_its_passage():
    """Each entry point of include/pcdn.h is preceded by a comment that cites the paper's passage
    defining the operation (Section, Eq., Algorithm, Appendix, Table, Lemma, Theorem), or says that
    it is library management with no passage, or that the paper has no counterpart."""
    import re
    with open(os.path.join(ROOT, "include", "pcdn.h")) as f:
        lines = f.read().split("\n")
    decl = re.compile(r"^(int|void|const char\*|int64_t)\s+(pcdn_\w+)\(")
    cite = re.compile(r"Section|Eq\.|Algorithm|Appendix|Table|Lemma|Theorem|no passage|no counterpart")
    seen = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j, block = i - 1, []
        while j >= 0 and (lines[j].strip().startswith(("/*", "*", "//")) or lines[j].strip().endswith("*/")):
            block.append(lines[j])
            j -= 1
        assert cite.search(" ".join(block)), m.group(2)
        seen.append(m.group(2))
    assert "pcdn_create" in seen and "pcdn_kkt" in seen and len(seen) >= 20
