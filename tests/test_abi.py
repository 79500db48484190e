"""Host-side checks of the C-ABI library (no GPU needed): it loads, it exports
every entry point include/cluster.h declares, argument errors come back as
status codes, and the host CSR builder is bit-identical to the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

pkg = pytest.importorskip("paper_2506_04045_b300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        names += re.findall(r"CLUSTER_API\s+[\w\s\*]*?\b(cluster_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    names = _declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    # exported dynamic symbols: nothing but the C ABI (hidden visibility otherwise)
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.lib_path()], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported
    assert all(e.startswith("cluster_") for e in exported if not e.startswith("_")), exported


def test_options_defaults():
    o = pkg.default_options()
    assert (o.precision, o.step_rule, o.stop_rule, o.accel, o.borrow, o.validate) == (0, 1, 0, 1, 0, 1)
    assert o.tau == 1.0 and o.tol == 0.0 and o.max_iter == 1000 and o.graph_chunk == 16
    assert o.fused_pass == 0 and o.relabel == 1 and o.l2_window == 1 and o.update_engine == 0 and o.overlap == 0


def test_init_argument_errors_are_status_codes():
    lib = pkg.load()
    ctx = ctypes.c_void_p()
    s = pkg.CSR()
    s.n, s.nnz, s.index64 = 10, 0, 1
    s.row_ptr = 0
    st = lib.cluster_init(ctypes.byref(s), 4, 0, None, None, ctypes.byref(ctx))
    assert st == pkg.EINVAL and "row_ptr" in pkg.last_error()
    s.row_ptr = 8
    st = lib.cluster_init(ctypes.byref(s), 0, 8, None, None, ctypes.byref(ctx))
    assert st == pkg.EINVAL and "k must be" in pkg.last_error()
    st = lib.cluster_init(ctypes.byref(s), 129, 8, None, None, ctypes.byref(ctx))
    assert st == pkg.EINVAL
    assert lib.cluster_step(None, 1, None) == pkg.EINVAL
    lib.cluster_destroy(None)


def _compare_builders(n, src, dst, w, diag):
    a = pkg.csr_from_edges(n, src, dst, w, diag)
    b = oracle.csr_from_edges(n, src, dst, w, diag)
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and np.array_equal(x, y)


@pytest.mark.parametrize("diag", [True, False])
def test_csr_builder_bit_exact_vs_oracle(diag):
    rng = np.random.default_rng(0)
    for n, m in [(1, 0), (1, 3), (7, 8), (50, 400), (300, 5000)]:
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        w = rng.random(m).astype(np.float32)
        _compare_builders(n, src, dst, w, diag)
        _compare_builders(n, src, dst, None, diag)


def test_csr_builder_matches_generator_assembly():
    # the synthetic generator's CSR equals the library's builder on the same edges
    s, d = synth.dcsbm_edges(3000, 8, 12.0, seed=5)
    rp, c, v = synth.assemble_csr(3000, s, d, seed=5)
    w = synth.pair_weights(s, d, 3000, 5).numpy()
    a = pkg.csr_from_edges(3000, s.numpy(), d.numpy(), w, True)
    assert np.array_equal(a[0], rp.numpy()) and np.array_equal(a[1], c.numpy()) and np.array_equal(a[2], v.numpy())


def test_csr_builder_errors():
    with pytest.raises(pkg.ClusterError) as ei:
        pkg.csr_from_edges(3, [0], [3])
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.ClusterError):
        pkg.csr_from_edges(3, [0], [1], [np.inf])


def test_ctypes_structs_match_the_c_header():
    # the binding's ctypes mirrors of the header's structs: same size, and every
    # named field at the same offset (a field added on one side only would shift
    # the ones after it and pass garbage through the ABI)
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2506_04045_b300 import binding as b
    pairs = {"cluster_csr": b.CSR, "cluster_options": b.Options, "cluster_report": b.Report,
             "cluster_kernel_times": b.KernelTimes, "cluster_server_options": b.ServerOptions,
             "cluster_server_stats": b.ServerStats, "cluster_request_times": b.RequestTimes}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cluster.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            if not fname.startswith("_"):
                lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as td:
        src, exe = os.path.join(td, "layout.c"), os.path.join(td, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    for cname, cls in pairs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            if not fname.startswith("_"):
                assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
