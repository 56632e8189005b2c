"""The library is usable from plain C and C++ through include/litevoxel.h
alone: a C program linked against liblitevoxel.so calls the host-only entry
points and argument checks (no device pointer is passed, so nothing can
launch), and the header compiles as C++ with its extern "C" block."""
import os
import shutil
import subprocess
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

PROGRAM = textwrap.dedent(r"""
    #include <math.h>
    #include <stdio.h>
    #include <string.h>
    #include "litevoxel.h"

    #define CHECK(c) do { if (!(c)) { printf("failed: %s (line %d)\n", #c, __LINE__); return 1; } } while (0)

    int main(void) {
      CHECK(lv_version() == ((LV_VERSION_MAJOR << 16) | LV_VERSION_MINOR));

      /* a(t) = clip((t - t0) / (t1 - t0), 0, 1) in ppm */
      CHECK(lv_prune_anneal_ppm(5.0, 0.0, 10.0) == 500000);
      CHECK(lv_prune_anneal_ppm(-1.0, 0.0, 10.0) == 0);
      CHECK(lv_prune_anneal_ppm(20.0, 0.0, 10.0) == 1000000);
      CHECK(lv_prune_anneal_ppm(3.0, 5.0, 5.0) == 1000000);

      /* Eq. 9: gamma ramps linearly from 0 at t0 to gamma_max at t1 */
      lv_lf_params lf;
      memset(&lf, 0, sizeof(lf));
      lf.eps = 1e-3f; lf.gamma_max = 0.8f; lf.t0 = 100.f; lf.t1 = 300.f; lf.pctl_ppm = 990000;
      CHECK(lv_lf_gamma(50.f, &lf) == 0.f);
      CHECK(fabsf(lv_lf_gamma(200.f, &lf) - 0.4f) < 1e-6f);
      CHECK(lv_lf_gamma(1000.f, &lf) == 0.8f);

      lv_camera cam;
      memset(&cam, 0, sizeof(cam));
      cam.width = 1237; cam.height = 822; cam.fx = cam.fy = 1071.f; cam.cx = 618.5f; cam.cy = 411.f;
      cam.w2c[0] = cam.w2c[5] = cam.w2c[10] = 1.f; cam.z_near = 0.05f;
      lv_raster_opts o;
      memset(&o, 0, sizeof(o));
      o.tile = 16; o.batch = 32; o.t_stop = 1e-4f;
      size_t ws = lv_forward_workspace_size(2000000, &cam, 1, &o, 10000000);
      CHECK(ws > (size_t)10000000 * 16);
      CHECK(lv_forward_workspace_size(2000000, &cam, 0, &o, 0) == 0);
      CHECK(lv_train_workspace_size() > 0);
      int32_t w[2] = {1237, 640}, h[2] = {822, 480};
      CHECK(lv_lf_workspace_size(w, h, 2) > lv_lf_workspace_size(w, h, 1));

      /* argument checks: null pointers and bad sizes are refused before anything runs */
      lv_voxels v;
      memset(&v, 0, sizeof(v));
      lv_fwd_out out;
      memset(&out, 0, sizeof(out));
      CHECK(lv_rasterize_forward(NULL, &cam, 1, &o, &out, NULL, 0, 0, NULL, NULL) == LV_ERR_INVALID_ARG);
      CHECK(strlen(lv_last_error()) > 0);
      CHECK(lv_rasterize_forward(&v, &cam, 1, &o, &out, NULL, 0, 0, NULL, NULL) == LV_ERR_INVALID_ARG);
      o.tile = 32; o.batch = 128;
      CHECK(lv_rasterize_forward(&v, &cam, 1, &o, &out, NULL, 0, 0, NULL, NULL) == LV_ERR_UNSUPPORTED);
      CHECK(lv_reset_stats(-1, NULL, NULL, NULL, NULL, NULL) == LV_ERR_INVALID_ARG);
      CHECK(lv_check_status(NULL, NULL) == LV_ERR_INVALID_ARG);
      lv_prune_params pp;
      memset(&pp, 0, sizeof(pp));
      CHECK(lv_prune_depth_quantile(10, NULL, NULL, NULL, NULL, NULL, &pp, NULL, NULL, NULL, 0, NULL, NULL) ==
            LV_ERR_INVALID_ARG);
      CHECK(lv_compact(NULL, NULL, NULL, 0, NULL, NULL, NULL, 0, NULL, NULL) == LV_ERR_INVALID_ARG);
      CHECK(lv_launch_count() == 0);
      printf("ok\n");
      return 0;
    }
""")


@pytest.fixture(scope="module")
def lib_dir():
    from paper_2511_02510_gb300 import build as B
    return os.path.dirname(B.build())


def test_c_program_links_and_calls_the_library(lib_dir, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src, exe = tmp_path / "consumer.c", tmp_path / "consumer"
    src.write_text(PROGRAM)
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", INC, str(src), "-o", str(exe), "-L", lib_dir,
                    "-llitevoxel", f"-Wl,-rpath,{lib_dir}", "-lm"], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_header_compiles_as_cxx(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    src = tmp_path / "h.cpp"
    src.write_text('#include "litevoxel.h"\nstatic_assert(sizeof(lv_camera) == 76, "camera layout: 19 four-byte fields");\n'
                   "int main() { return lv_version() < 0; }\n")
    subprocess.run([cxx, "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", INC, str(src)], check=True,
                   capture_output=True)
