"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/vos.h declares, and the ctypes structures
match the C layout (checked with a gcc-compiled probe)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vos.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vos_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_07019_gb300 import build_lib, vos
    build_lib.build()
    return vos.load_library()


def test_header_declares_the_step_api():
    names = _declared()
    for n in ("vos_create", "vos_step", "vos_fields", "vos_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2204_07019_gb300 import vos
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(vos.EXPORTED_SYMBOLS) == names


def test_binding_has_every_declared_call_under_its_name():
    """The Python binding offers each C entry point under the same name."""
    from paper_2204_07019_gb300 import vos
    names = _declared()
    missing = [n for n in names if not callable(getattr(vos, n, None)) or n not in vos.__all__]
    assert not missing, missing


def test_batch_handle_rejects_bad_index_without_gpu():
    from paper_2204_07019_gb300 import vos
    with pytest.raises(vos.VosError):
        vos.vos_batch_handle(None, 0)


def test_struct_layout_matches_c(tmp_path):
    from paper_2204_07019_gb300 import vos
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "vos.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(vos_params),'
                   ' sizeof(vos_stats), sizeof(vos_device_fields), sizeof(vos_allocator),'
                   ' offsetof(vos_params, p_rtol), offsetof(vos_params, wall_mask),'
                   ' offsetof(vos_stats, status) + offsetof(vos_stats, rmax));return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(vos.VosParams), ctypes.sizeof(vos.VosStats), ctypes.sizeof(vos.VosDeviceFields),
            ctypes.sizeof(vos.VosAllocator), vos.VosParams.p_rtol.offset, vos.VosParams.wall_mask.offset,
            vos.VosStats.status.offset + vos.VosStats.rmax.offset]
    assert got == want


def test_invalid_parameters_rejected_without_gpu(lib):
    """vos_create validates before touching the device: bad sizes fail with
    VOS_EINVAL and a message."""
    import numpy as np
    from paper_2204_07019_gb300 import inputs as I, vos
    es = np.zeros((1, 4, 4))
    for bad in (dict(dim=4), dict(nx=1), dict(eps_min=0.0), dict(method=7), dict(p_rtol=2.0),
                dict(flow_subiters=0), dict(qs_rtol=-1.0)):
        prm = I.make_params(es.shape, Pe=1, Da=1, L=1, **bad)
        with pytest.raises(vos.VosError) as ei:
            vos.vos_create(es, prm, allocator="cuda")
        assert ei.value.code == vos.VOS_EINVAL
        assert vos.vos_last_error()
    prm = I.make_params(es.shape, Pe=1, Da=1, L=1)
    with pytest.raises(vos.VosError):
        vos.vos_create(es + 2.0, prm, allocator="cuda")


def test_other_entry_points_reject_bad_arguments_without_gpu(lib):
    """Entry points that validate before any CUDA call: the FP64-quotient
    check, the tensor-core convolution and the U-Net constructor return
    VOS_EINVAL with a message (n = 0 is a no-op)."""
    import ctypes as C
    from paper_2204_07019_gb300 import vos
    assert lib.vos_fp64_div_check(None, None, -1, None, None) == vos.VOS_EINVAL
    assert lib.vos_fp64_div_check(None, None, 0, None, None) == vos.VOS_OK
    assert lib.vos_fp64_div_check(None, None, 5, None, None) == vos.VOS_EINVAL
    assert b"NULL" in lib.vos_last_error(None)
    # cin not a multiple of 8, cout out of [16, 96] or not a multiple of 16, no output
    dummy = C.c_void_p(16)
    for cin, cout, y in ((12, 16, dummy), (8, 8, dummy), (8, 112, dummy), (8, 24, dummy), (8, 16, None)):
        rc = lib.vos_conv3d_bf16(dummy, 4, 4, 4, cin, dummy, None, cout, 0, y, None, None)
        assert rc == vos.VOS_EINVAL, (cin, cout)
    assert b"vos_conv3d_bf16" in lib.vos_last_error(None)
    out = C.c_void_p()
    assert lib.vos_unet_create(3, 8, 8, 0, None, C.byref(out)) == vos.VOS_EINVAL
    assert lib.vos_unet_create(2048, 2048, 2048, 0, None, C.byref(out)) == vos.VOS_EINVAL
    assert not out.value


def test_noalloc_dt_rejects_bad_arguments_without_gpu(lib):
    """vos_suggest_dt_noalloc checks its arguments before any CUDA call:
    nx < 2, a missing v array on a grid with ny > 1 (v may only be NULL when
    ny == 1) and a missing w array in 3D are refused with VOS_EINVAL."""
    import ctypes as C
    from paper_2204_07019_gb300 import inputs as I, vos
    d = C.c_void_p(256)
    out = C.c_double(-1.0)
    # (grid shape (nz, ny, nx), v, w): nx < 2; ny > 1 without v; 3D without w
    cases = (((1, 4, 1), d, None), ((1, 4, 8), None, None), ((3, 4, 8), d, None))
    for shape, v, w in cases:
        ps = vos._params_struct(I.make_params(shape, Pe=1, Da=1, L=1))
        rc = lib.vos_suggest_dt_noalloc(C.byref(ps), d, d, v, w, d, 0.5, 0.005, None, C.byref(out))
        assert rc == vos.VOS_EINVAL, shape
        assert b"vos_suggest_dt_noalloc" in lib.vos_last_error(None)
    assert out.value == -1.0
