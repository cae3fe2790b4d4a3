"""The C-ABI library loads and exports every entry point that include/svt.h and include/svt_serve.h
declare (no GPU work: nothing here launches a kernel).  Also checks the binding's prototypes cover
the headers."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", "svt.h"), os.path.join(ROOT, "include", "svt_serve.h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(svt_[a-z_A-Z0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_0810_3286_gb300 import build
    return build.build()


def test_header_declares_expected_calls():
    names = _declared()
    for required in ["svt_create", "svt_step", "svt_solve", "svt_get_factors", "svt_configure", "svt_destroy",
                     "svt_get_Y", "svt_save_state", "svt_load_state", "svt_sample_omega", "svt_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(svt_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_header(libpath):
    from paper_0810_3286_gb300 import _abi
    L = _abi.load(libpath)
    for name in _declared():
        assert hasattr(L, name)
        assert name in _abi.PROTOTYPES, name
    # host-only calls that do not touch the GPU
    import ctypes
    opt = _abi.svt_options()
    L.svt_default_options(ctypes.byref(opt))
    assert opt.ell == 5 and opt.k_max == 1000 and opt.precision == _abi.SVT_FP64
    assert L.svt_kernel_launches(None) == 0


def test_create_rejects_bad_arguments_before_any_device_work(libpath):
    """Argument validation happens on the host before the library touches a device."""
    import ctypes
    import numpy as np
    from paper_0810_3286_gb300 import _abi
    L = _abi.load(libpath)
    rows = np.zeros(3, np.int32)
    ctx = ctypes.c_void_p()
    st = L.svt_create(0, 5, 3, rows.ctypes.data, rows.ctypes.data, rows.ctypes.data, None, ctypes.byref(ctx))
    assert st == _abi.SVT_ERR_ARG and not ctx.value
    st = L.svt_create(4, 5, 21, rows.ctypes.data, rows.ctypes.data, rows.ctypes.data, None, ctypes.byref(ctx))
    assert st == _abi.SVT_ERR_ARG
    assert b"nnz" in L.svt_last_error(None)
    # option checks come before any device work too
    opt = _abi.svt_options()
    L.svt_default_options(ctypes.byref(opt))
    assert opt.orth_grid == 0 and opt.lanczos_tol == 0.0
    opt.orth_grid = -1
    st = L.svt_create(4, 5, 3, rows.ctypes.data, rows.ctypes.data, rows.ctypes.data, ctypes.byref(opt),
                      ctypes.byref(ctx))
    assert st == _abi.SVT_ERR_ARG and b"orth_grid" in L.svt_last_error(None)
    opt.orth_grid = 0
    opt.precision = 7
    st = L.svt_create(4, 5, 3, rows.ctypes.data, rows.ctypes.data, rows.ctypes.data, ctypes.byref(opt),
                      ctypes.byref(ctx))
    assert st == _abi.SVT_ERR_ARG and b"precision" in L.svt_last_error(None)


def test_binding_struct_layouts_match_the_headers(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that a C compiler gives
    the header's struct (a field added on one side only would shift the ones after it)."""
    import ctypes
    import shutil
    from paper_0810_3286_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [_abi.svt_options, _abi.svt_step_info, _abi.svt_result, _abi.svt_batch_options, _abi.svt_server_options, _abi.svt_job,
               _abi.svt_job_result, _abi.svt_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "svt.h"', '#include "svt_serve.h"',
             'int main(void) {']
    for s in structs:
        name = s.__name__
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in s._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append('  return 0;\n}')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for s in structs:
        name = s.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(s), name
        for f, _ in s._fields_:
            assert got[(name, f)] == getattr(s, f).offset, (name, f)


def test_batch_rejects_bad_batches_before_any_device_work(libpath):
    """svt_batch_solve checks the job count and its output arrays on the host first."""
    import ctypes
    from paper_0810_3286_gb300 import _abi
    L = _abi.load(libpath)
    opt = _abi.svt_batch_options()
    L.svt_batch_default_options(ctypes.byref(opt))
    assert (opt.spmm_grid, opt.update_grid, opt.autotune, opt.concurrent) == (0, 0, 0, 1)
    res = (_abi.svt_result * 33)()
    st = (ctypes.c_int * 33)()
    jobs = (ctypes.c_void_p * 33)()
    for n in (0, 33):   # 1 <= n <= 32
        assert L.svt_batch_solve(ctypes.cast(jobs, ctypes.c_void_p), n, None, None, 1e-4, 27, ctypes.byref(opt),
                                 ctypes.cast(res, ctypes.c_void_p), ctypes.cast(st, ctypes.c_void_p)) == _abi.SVT_ERR_ARG
    # missing outputs, and a NULL context in the list
    assert L.svt_batch_solve(ctypes.cast(jobs, ctypes.c_void_p), 2, None, None, 1e-4, 27, None, None,
                             ctypes.cast(st, ctypes.c_void_p)) == _abi.SVT_ERR_ARG
    assert L.svt_batch_solve(ctypes.cast(jobs, ctypes.c_void_p), 2, None, None, 1e-4, 27, None,
                             ctypes.cast(res, ctypes.c_void_p), ctypes.cast(st, ctypes.c_void_p)) == _abi.SVT_ERR_ARG
