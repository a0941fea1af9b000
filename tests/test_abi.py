"""CPU-side checks of the C ABI: the library exports every symbol the headers under include/
declare and rejects bad descriptors before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ohm_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libohm():
    from paper_1009_0798_gb300 import build
    build.build()
    from paper_1009_0798_gb300 import ohm
    return ohm


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("ohm_create_hierarchy", "ohm_set_eta", "ohm_cn_step", "ohm_residual_norm", "ohm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libohm):
    L = C.CDLL(libohm.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(libohm):
    assert libohm.status_string(libohm.OHM_OK) == "ok"
    assert "converged" in libohm.status_string(libohm.OHM_ERR_NOT_CONVERGED)


def _desc(libohm, base=(16, 16, 16), blocks=None, **kw):
    from paper_1009_0798_gb300 import workloads as W
    h = W.uniform(*base, 1.0 / base[0])
    return h.blocks if blocks is None else blocks


@pytest.mark.parametrize("case", ["bad_base", "unsorted", "duplicate", "incomplete_base", "bad_lambda",
                                  "bad_counts", "not_nested", "incomplete_octet", "krylov_fp64", "bad_precision", "omega_2", "omega_negative", "coarse_nu_negative",
                                  "bad_inner_tol"])
def test_invalid_descriptors_are_rejected_without_gpu(libohm, case):
    from paper_1009_0798_gb300 import workloads as W
    kw = dict(lam=0.5, nu_pre=2, nu_post=2, n_coarse=8, max_outer=10, stream=0)
    base = (16, 16, 16)
    blocks = W.uniform(16, 16, 16, 1.0 / 16).blocks.copy()
    if case == "bad_base":
        base = (12, 16, 16)
    elif case == "unsorted":
        h = W.refined(16, 16, 16, 1.0 / 16, [lambda lo, hi: lo[0] < 0.3])
        blocks = h.blocks[::-1].copy()
    elif case == "duplicate":
        blocks = np.concatenate([blocks, blocks[:1]])
    elif case == "incomplete_base":
        blocks = blocks[:-1]
    elif case == "bad_lambda":
        kw["lam"] = 0.0
    elif case == "bad_counts":
        kw["n_coarse"] = 0
    elif case == "krylov_fp64":  # float64 FGMRES is for single problems only
        kw.update(krylov=4, n_instances=2)
    elif case == "bad_inner_tol":
        kw.update(precision=libohm.OHM_MIXED, inner_tol=1.5)
    elif case == "bad_precision":
        kw["precision"] = libohm.OHM_MIXED_FF_CHECKED + 1
    elif case == "omega_2":
        kw["omega"] = 2.0
    elif case == "omega_negative":
        kw["omega"] = -0.5
    elif case == "coarse_nu_negative":
        kw["nu_coarse"] = (-1, 1)
    elif case == "not_nested":
        # a level-2 octet whose parent's neighbourhood is missing at level 1
        h = W.refined(32, 32, 32, 1.0 / 32, [lambda lo, hi: lo[0] < 0.2 and lo[1] < 0.2 and lo[2] < 0.2])
        extra = np.array([[2, 0, 0, 0], [2, 1, 0, 0], [2, 0, 1, 0], [2, 1, 1, 0],
                          [2, 0, 0, 1], [2, 1, 0, 1], [2, 0, 1, 1], [2, 1, 1, 1]], np.int32)
        blocks = np.concatenate([h.blocks, extra])
    elif case == "incomplete_octet":
        h = W.refined(16, 16, 16, 1.0 / 16, [lambda lo, hi: lo[0] < 0.3])
        blocks = h.blocks[:-1].copy()
    with pytest.raises(libohm.OhmError) as ei:
        libohm.ohm_create_hierarchy(base, 1.0 / base[0], blocks, **kw)
    assert ei.value.status == libohm.OHM_ERR_INVALID


def test_batch_bytes_grow_with_instances(libohm):
    """ohm_hierarchy_bytes: host-only sizing of batched hierarchies (admission control)."""
    from paper_1009_0798_gb300 import workloads as W
    h = W.uniform(16, 16, 16, 1.0 / 16)
    one = libohm.ohm_hierarchy_bytes(h.base_cells, h.dx0, h.blocks, precision=libohm.OHM_MIXED, n_instances=1)
    four = libohm.ohm_hierarchy_bytes(h.base_cells, h.dx0, h.blocks, precision=libohm.OHM_MIXED, n_instances=4)
    assert 3.5 * one < four < 4.5 * one
    kry = libohm.ohm_hierarchy_bytes(h.base_cells, h.dx0, h.blocks, precision=libohm.OHM_MIXED, n_instances=4, krylov=4)
    assert kry > four  # Krylov basis and per-instance product scratch
    with pytest.raises(libohm.OhmError):
        libohm.ohm_hierarchy_bytes(h.base_cells, h.dx0, h.blocks, n_instances=4, krylov=4)  # no batched FP64 Krylov


def test_server_rejects_bad_descriptor_without_gpu(libohm):
    from paper_1009_0798_gb300 import server
    with pytest.raises(libohm.OhmError):
        server.Server(hbm_budget_bytes=0)
    with pytest.raises(libohm.OhmError):
        server.Server(hbm_budget_bytes=1 << 30, max_batch=0)


def test_ctypes_mirrors_match_the_c_layouts(tmp_path):
    """The Python structures that mirror ohm_hier_desc, ohm_tune_result, ohm_step_stats,
    ohm_server_desc and ohm_request have the sizes and field offsets the C compiler gives the
    header's structs."""
    import ctypes as C
    import shutil
    import subprocess
    from paper_1009_0798_gb300 import ohm, server
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    mirrors = {"ohm_hier_desc": ohm.HierDesc, "ohm_tune_result": ohm.TuneResult, "ohm_step_stats": ohm.StepStats,
               "ohm_server_desc": server.ServerDesc, "ohm_request": server.Request}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ohm_server.h"', "int main(void) {"]
    cnames = {"lam": "lambda"}
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {cnames.get(f, f)}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.split("\n") if l)
    for cname, py in mirrors.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
