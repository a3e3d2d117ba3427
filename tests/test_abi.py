"""Host-side checks of the C ABI (no GPU needed): libgs.so loads, exports every
function include/gs.h declares, and rejects bad arguments synchronously before
touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def A():
    from paper_2403_16095_b300.build import build
    build()
    from paper_2403_16095_b300 import _abi
    return _abi


def test_every_declared_symbol_is_exported(A):
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(A.lib, n), n
    assert set(names) == set(A.EXPORTS)


def test_header_compiles_as_plain_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "gs.h"\nint main(void){ return gs_abi_version() == GS_ABI_VERSION ? 0 : 1; }\n')
    lib = os.path.join(ROOT, "paper_2403_16095_b300", "lib")
    r = os.system(f"gcc -std=c99 -Wall -Werror -I{ROOT}/include {src} -L{lib} -lgs -Wl,-rpath,{lib} "
                  f"-o {tmp_path}/t && {tmp_path}/t")
    assert r == 0


def test_pure_host_queries(A):
    assert A.lib.gs_abi_version() == A.ABI_VERSION == 9
    assert A.gs_bin_tiles_workspace_size(1000, 5000) >= 5000 * (8 + 8)
    assert A.gs_bin_tiles_workspace_size(10, 0) == 0
    cams = [type("C", (), dict(width=640, height=480, fx=600, fy=600, cx=320, cy=240, znear=0.2))()]
    assert A.gs_pose_partials_per_frame(A.GS_MODE_POSE, 10, cams, 16) == 1200
    assert A.gs_pose_partials_per_frame(A.GS_MODE_FULL, 1000, cams, 16) == 4
    assert A.gs_render_bwd_workspace_size(100, A.GS_MODE_FULL) >= 100 * 12 * 4


def test_argument_errors_are_synchronous(A):
    lib = A.lib
    opts = A.gs_opts(16, A.GS_MODE_POSE, 1.3, 0.0)
    cam = (A.gs_camera * 1)(A.gs_camera(64, 48, 50.0, 50.0, 32.0, 24.0, 0.2))
    g = A.gs_gaussians(10, None, None, None, None, None, None)
    proj = A.gs_projected(10, 1, None, None, None)
    st = lib.gs_project(C.byref(g), 1, cam, None, C.byref(opts), C.byref(proj), None, None)
    assert st == A.GS_ERR_INVALID_ARG and "NULL" in A.last_error()
    bad_tile = A.gs_opts(12, A.GS_MODE_FWD, 1.3, 0.0)
    g0 = A.gs_gaussians(0, None, None, None, None, None, None)
    p0 = A.gs_projected(0, 1, None, None, None)
    st = lib.gs_project(C.byref(g0), 1, cam, C.c_void_p(16), C.byref(bad_tile), C.byref(p0), C.c_void_p(16), None)
    assert st == A.GS_ERR_INVALID_ARG and "tile" in A.last_error()
    st = lib.gs_project(C.byref(g0), 0, cam, C.c_void_p(16), C.byref(opts), C.byref(p0), C.c_void_p(16), None)
    assert st == A.GS_ERR_INVALID_ARG and "n_frames" in A.last_error()
    many = (A.gs_camera * (A.GS_MAX_FRAMES + 1))(*[A.gs_camera(64, 48, 50.0, 50.0, 32.0, 24.0, 0.2)] * (A.GS_MAX_FRAMES + 1))
    st = lib.gs_project(C.byref(g0), A.GS_MAX_FRAMES + 1, many, C.c_void_p(16), C.byref(opts), C.byref(p0),
                        C.c_void_p(16), None)
    assert st == A.GS_ERR_INVALID_ARG and "n_frames" in A.last_error()
    badcam = (A.gs_camera * 1)(A.gs_camera(0, 48, 50.0, 50.0, 32.0, 24.0, 0.2))
    st = lib.gs_project(C.byref(g0), 1, badcam, C.c_void_p(16), C.byref(opts), C.byref(p0), C.c_void_p(16), None)
    assert st == A.GS_ERR_INVALID_ARG
    # POSE mode without a Jacobian buffer (rejected before any launch; with no
    # Gaussians there is nothing to write and NULL is accepted)
    p = C.c_void_p(256)
    g10 = A.gs_gaussians(10, p, p, p, p, p, p)
    p10 = A.gs_projected(10, 1, p, p, None)
    st = lib.gs_project(C.byref(g10), 1, cam, C.c_void_p(16), C.byref(opts), C.byref(p10), C.c_void_p(16), None)
    assert st == A.GS_ERR_INVALID_ARG and "pose_jac" in A.last_error()
    # backward needs POSE or FULL
    fwd_opts = A.gs_opts(16, A.GS_MODE_FWD, 1.3, 0.0)
    tiles = A.gs_tiles(10, 12, C.c_void_p(256), None, C.c_void_p(256))
    img = A.gs_image()
    st = lib.gs_render_bwd(C.byref(p0), C.byref(tiles), 1, cam, None, None, None, C.byref(img), None, None,
                           C.byref(fwd_opts), None, None, None, None, None, 0, None)
    assert st == A.GS_ERR_INVALID_ARG and "POSE or FULL" in A.last_error()
    # workspace too small
    ws_opts = A.gs_opts(16, A.GS_MODE_POSE, 1.3, 0.0)
    st = lib.gs_bin_tiles(C.byref(p0), 1, cam, C.byref(ws_opts), C.byref(tiles), C.c_void_p(256), C.c_void_p(256), 8, None)
    assert st == A.GS_ERR_INVALID_ARG and "workspace" in A.last_error()
    st = lib.gs_pose_grad_reduce(None, 1, 1, None, None, None)
    assert st == A.GS_ERR_INVALID_ARG


def test_schedule_and_batch_options_are_checked(A):
    """gs_opts.batch must be 0, 256 or 512 and gs_opts.sched a known schedule;
    the persistent schedule needs the caller's work queue. All rejected before
    any launch."""
    lib = A.lib
    cam = (A.gs_camera * 1)(A.gs_camera(64, 48, 50.0, 50.0, 32.0, 24.0, 0.2))
    p = C.c_void_p(256)
    p0 = A.gs_projected(0, 1, p, p, None)
    img = A.gs_image(p, p, None, None, None, None, p, p)
    st32 = C.c_void_p(256)
    for bad, word in ((A.gs_opts(16, A.GS_MODE_FWD, 1.3, 0.0, 300, 0), "batch"),
                      (A.gs_opts(16, A.GS_MODE_FWD, 1.3, 0.0, 0, 7), "sched")):
        tiles = A.gs_tiles(10, 12, p, None, p)
        st = lib.gs_render_fwd(C.byref(p0), C.byref(tiles), 1, cam, None, C.byref(bad), C.byref(img), st32, None)
        assert st == A.GS_ERR_INVALID_ARG and word in A.last_error()
    persist = A.gs_opts(16, A.GS_MODE_FWD, 1.3, 0.0, 256, A.GS_SCHED_PERSISTENT)
    tiles = A.gs_tiles(10, 12, p, None, p)  # no queue
    st = lib.gs_render_fwd(C.byref(p0), C.byref(tiles), 1, cam, None, C.byref(persist), C.byref(img), st32, None)
    assert st == A.GS_ERR_INVALID_ARG and "queue" in A.last_error()


def test_tiles_touched_required_only_where_read(A):
    """The binning and the FULL backward read each record's tiles_touched; the
    blend calls read only rec and accept NULL there. Checked on the argument
    validation, which runs before any launch."""
    lib = A.lib
    cam = (A.gs_camera * 1)(A.gs_camera(64, 48, 50.0, 50.0, 32.0, 24.0, 0.2))
    p = C.c_void_p(256)
    no_touched = A.gs_projected(10, 1, p, None, p)
    tiles = A.gs_tiles(64, 12, p, None, p)
    status = C.c_void_p(256)
    # binning: rejected for the missing counts
    opts = A.gs_opts(16, A.GS_MODE_POSE, 1.3, 0.0)
    st = lib.gs_bin_tiles(C.byref(no_touched), 1, cam, C.byref(opts), C.byref(tiles), status, p, 1 << 20, None)
    assert st == A.GS_ERR_INVALID_ARG and "tiles_touched" in A.last_error()
    # FULL backward: rejected for the missing counts (before its other checks
    # of the forward images)
    full = A.gs_opts(16, A.GS_MODE_FULL, 1.3, 0.0)
    img = A.gs_image()
    st = lib.gs_render_bwd(C.byref(no_touched), C.byref(tiles), 1, cam, None, None, None, C.byref(img), None, None,
                           C.byref(full), None, None, None, status, p, 1 << 20, None)
    assert st == A.GS_ERR_INVALID_ARG and "tiles_touched" in A.last_error()
    # POSE backward: the counts are not read; it fails on the missing forward
    # images instead
    st = lib.gs_render_bwd(C.byref(no_touched), C.byref(tiles), 1, cam, None, None, None, C.byref(img), None, None,
                           C.byref(opts), None, None, None, status, p, 1 << 20, None)
    assert st == A.GS_ERR_INVALID_ARG and "tiles_touched" not in A.last_error()


def test_full_backward_binding_needs_touched(A):
    """The Python binding refuses a FULL-mode backward without tiles_touched
    before it marshals any tensor."""
    full = A.gs_opts(16, A.GS_MODE_FULL, 1.3, 0.0)
    with pytest.raises(ValueError, match="tiles_touched"):
        A.gs_render_bwd(10, [None], full, None, None, None, None, None, None, None, {}, None, None, None, None, None,
                        None, None)
