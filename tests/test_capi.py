"""The C-ABI library builds, loads and exports every entry point that
include/utf16wf.h declares; argument errors are rejected on the host before
any CUDA call (these tests run without a GPU and make no compute call)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for h in sorted(os.listdir(HEADER_DIR)):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(utf16_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def capi():
    from paper_2601_06349_gb300 import build
    build.build()
    import paper_2601_06349_gb300 as pkg
    return pkg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("utf16_to_well_formed", "utf16_to_well_formed_inplace", "utf16_is_well_formed",
                     "utf16_to_well_formed_batch", "utf16_to_well_formed_batch_inplace",
                     "utf16_is_well_formed_batch", "utf16_strerror", "utf16_to_well_formed_host"):
        assert required in names


def test_every_declared_symbol_is_exported(capi):
    missing = [n for n in declared_functions() if not hasattr(capi, n)]
    assert not missing, missing


def test_strerror(capi):
    import paper_2601_06349_gb300 as pkg
    for code in (0, -1, -2, -3, -4, -5, -6, -7, 12345):
        s = pkg.strerror(code)
        assert isinstance(s, str) and s


def test_argument_errors_before_any_cuda_call(capi):
    vp = ctypes.c_void_p
    # negative sizes
    assert capi.utf16_to_well_formed(vp(16), vp(4096), -1, None) == -1
    assert capi.utf16_to_well_formed_inplace(vp(16), -5, None) == -1
    # null buffers with n > 0
    assert capi.utf16_to_well_formed(None, vp(4096), 10, None) == -1
    assert capi.utf16_to_well_formed(vp(4096), None, 10, None) == -1
    assert capi.utf16_to_well_formed_inplace(None, 10, None) == -1
    # odd (not 2-byte aligned) buffers
    assert capi.utf16_to_well_formed(vp(4097), vp(8192), 10, None) == -1
    # partial overlap
    assert capi.utf16_to_well_formed(vp(4096), vp(4098), 10, None) == -2
    # missing first-error output
    assert capi.utf16_is_well_formed(vp(4096), 10, None, None) == -1
    assert capi.utf16_to_well_formed_first_bad(vp(4096), vp(8192), 10, None, None) == -1
    # batch: negative count, null offsets, misaligned offsets
    assert capi.utf16_to_well_formed_batch(vp(4096), vp(8192), vp(64), -1, None) == -1
    assert capi.utf16_to_well_formed_batch(vp(4096), vp(8192), None, 3, None) == -1
    assert capi.utf16_to_well_formed_batch(vp(4096), vp(8192), vp(65), 3, None) == -1
    assert capi.utf16_is_well_formed_batch(vp(4096), vp(64), 3, None, None) == -1
    # host entry point
    assert capi.utf16_to_well_formed_host(None, None, 3, None) == -1
    # offsets check and histogram tuning
    assert capi.utf16_check_offsets(None, 3, vp(4096), None) == -1
    assert capi.utf16_check_offsets(vp(64), -1, vp(4096), None) == -1
    hist = (ctypes.c_int64 * 4)(0, 1, 2, 3)
    assert capi.utf16_autotune(2, hist, 4) == -1
    assert capi.utf16_autotune(0, None, 4) == -1
    assert capi.utf16_autotune(0, hist, 0) == -1
    assert capi.utf16_autotune(1, hist, 65) == -1
    bad = (ctypes.c_int64 * 2)(5, -1)
    assert capi.utf16_autotune(1, bad, 2) == -1


def test_empty_inputs_are_noops(capi):
    vp = ctypes.c_void_p
    assert capi.utf16_to_well_formed(None, None, 0, None) == 0
    assert capi.utf16_to_well_formed_inplace(None, 0, None) == 0
    assert capi.utf16_to_well_formed_batch(None, None, None, 0, None) == 0
    assert capi.utf16_to_well_formed_batch_inplace(None, None, 0, None) == 0
    fb = ctypes.c_int64(-1)
    assert capi.utf16_to_well_formed_host(None, None, 0, ctypes.addressof(fb)) == 0
    assert fb.value == 0


def test_binding_rejects_cpu_tensors(capi):
    torch = pytest.importorskip("torch")
    import paper_2601_06349_gb300 as pkg
    with pytest.raises(ValueError):
        pkg.to_well_formed(torch.zeros(4, dtype=torch.int16))
    with pytest.raises(TypeError):
        pkg.to_well_formed(torch.zeros(4, dtype=torch.float32))


def test_checked_mode_switch(capi):
    """utf16_set_checked / utf16_get_checked need no GPU; the initial value
    comes from UTF16WF_CHECKED."""
    import subprocess
    import sys
    import paper_2601_06349_gb300 as pkg
    was = pkg.get_checked()
    try:
        pkg.set_checked(True)
        assert capi.utf16_get_checked() == 1
        pkg.set_checked(False)
        assert not pkg.get_checked()
    finally:
        pkg.set_checked(was)
    code = "import paper_2601_06349_gb300 as p; print(p.get_checked())"
    for env_value, want in (("1", "True"), ("0", "False"), ("", "False")):
        env = dict(os.environ, UTF16WF_CHECKED=env_value)
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=120)
        assert out.returncode == 0, out.stderr
        assert out.stdout.strip() == want, (env_value, out.stdout)


def test_server_default_options_match_the_header(capi):
    """utf16_server_default_options needs no GPU; its values are the ones the
    header documents."""
    import paper_2601_06349_gb300 as pkg
    o = pkg.ServerOptions()
    assert capi.utf16_server_default_options(ctypes.byref(o)) == 0
    assert (o.hbm_budget_bytes, o.max_batch_strings, o.max_batch_bytes, o.max_inflight_batches,
            o.staging_bytes, o.small_request_bytes, o.inject_fail_mod, o.direct_host_access,
            o.inject_copy_fail_mod, o.inject_copy_fail_step) == \
        (4 << 30, 1 << 16, 16 << 20, 8, 32 << 20, 256 << 10, 0, 0, 0, 0)
    text = open(os.path.join(HEADER_DIR, "utf16wf.h")).read()
    assert "16 MiB packed per batch, 8 slots, 32 MiB staging" in text


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes through the C ABI has the header's
    size and field offsets (a C program built with gcc against
    include/utf16wf.h prints them)."""
    import ctypes
    import shutil
    import subprocess
    import paper_2601_06349_gb300 as pkg
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    pairs = {"utf16_config": pkg.Config, "utf16_server_options": pkg.ServerOptions,
             "utf16_completion": pkg.Completion, "utf16_server_stats": pkg.ServerStats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "utf16wf.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = {}
    for line in got:
        if line:
            cname, field, value = line.split()
            seen[(cname, field)] = int(value)
    for cname, py in pairs.items():
        assert seen[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert seen[(cname, field)] == getattr(py, field).offset, (cname, field)
