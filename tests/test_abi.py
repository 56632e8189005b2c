"""The C-ABI library loads without a GPU and exports every function the header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "litevoxel.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(lv_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_02510_gb300 import build as B
    return ctypes.CDLL(B.build())


def test_header_declares_the_calls():
    names = declared_functions()
    for n in ("lv_rasterize_forward", "lv_rasterize_backward", "lv_prune_depth_quantile", "lv_subdivide_priority",
              "lv_lf_weighted_loss", "lv_unpack_wmax"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2511_02510_gb300 import litevoxel as L
    assert set(declared_functions()) <= set(L.SIGNATURES)


def test_host_only_queries_work_without_gpu(lib):
    from paper_2511_02510_gb300 import litevoxel as L
    from paper_2511_02510_gb300 import synth
    L.load()
    assert L.load().lv_version() == (0 << 16) | 1
    cams = L.make_cameras([synth.orbit_camera(128, 96, 60.0, 3.0, 0.0, 10.0)])
    opts = L.make_opts()
    a = L.lv_forward_workspace_size(1000, cams, 1, opts, 0)
    b = L.lv_forward_workspace_size(1000, cams, 1, opts, 10000)
    # a pair of the capacity costs 16 bytes, (tile, slot) in two ping-pong buffers, plus the sort's
    # look-back words (two 8-byte words per digit value and 2048 items: 2 bytes per pair)
    assert a > 0 and a + 10000 * 16 <= b <= a + 10000 * 18 + 8192
    assert L.lv_forward_workspace_size(1000, cams, 0, opts, 0) == 0


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library every call raises: there is no CPU fallback (checked in a child process
    whose binding points at a path that does not exist)."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2511_02510_gb300 import litevoxel as L\n"
        "L.LIB_PATH = %r\n"
        "try:\n"
        "    L.lv_prune_anneal_ppm(1.0, 0.0, 2.0)\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n" % (ROOT, str(tmp_path / "nowhere" / "liblitevoxel.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "missing" in r.stdout, r.stdout + r.stderr
