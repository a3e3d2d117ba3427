"""gs_bin_tiles_noalloc: the binning entry point for callers that cannot
allocate device memory (a real-time tracking thread that must not block on the
allocator, a process whose device memory belongs to another framework's pool,
a plug-in limited to memory declared at load time). It uses a static device
scratch array instead of a caller workspace; this test calls it through the
C ABI twice in a row, on different inputs, and checks every output against
gs_bin_tiles with a caller workspace (integer outputs: bit-exact)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _records(n, cam, tile, seed):
    rng = np.random.default_rng(seed)
    x0 = rng.integers(0, cam.width, n)
    y0 = rng.integers(0, cam.height, n)
    rect = np.c_[x0, y0, np.minimum(cam.width - 1, x0 + rng.integers(0, 60, n)),
                 np.minimum(cam.height - 1, y0 + rng.integers(0, 60, n))].astype(np.int32)
    rect[rng.uniform(size=n) < 0.1] = [1, 1, 0, 0]
    rec = np.zeros((n, 16), np.float32)
    rec[:, 6] = rng.choice(np.float32([0.5, 1.25, 2.0, 3.5, 9.0]), n)
    rec.view(np.int32)[:, 12:16] = rect
    ok = rect[:, 0] <= rect[:, 2]
    touched = np.where(ok, (rect[:, 2] // tile - rect[:, 0] // tile + 1) * (rect[:, 3] // tile - rect[:, 1] // tile + 1), 0)
    return torch.from_numpy(rec.reshape(-1)).cuda(), torch.from_numpy(touched.astype(np.int32)).cuda(), int(touched.sum())


def _bin(A, use_noalloc, n, cam, opts, rec, touched, cap):
    n_tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    values = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    keys = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    ranges = torch.full((2 * n_tiles,), -1, dtype=torch.int32, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    if use_noalloc:
        A.gs_bin_tiles_noalloc(n, [cam], opts, rec, touched, values, keys, ranges, status)
    else:
        ws = torch.empty(A.gs_bin_tiles_workspace_size(n, cap), dtype=torch.uint8, device="cuda")
        A.gs_bin_tiles(n, [cam], opts, rec, touched, values, keys, ranges, status, ws)
    torch.cuda.synchronize()
    return values.cpu(), keys.cpu(), ranges.cpu(), status.cpu()


def test_noalloc_binning_matches_workspace_binning_on_two_calls():
    from paper_2403_16095_b300 import _abi as A
    cam = synth.Camera(640, 480, 600.0, 600.0, 320.0, 240.0)
    opts = A.gs_opts(16, A.GS_MODE_POSE, 1.3, 0.0)
    for call, (n, seed) in enumerate([(20_000, 11), (7_000, 12)]):
        rec, touched, P = _records(n, cam, 16, seed)
        cap = P + 100
        assert cap <= A.GS_NOALLOC_MAX_PAIRS
        want = _bin(A, False, n, cam, opts, rec, touched, cap)
        got = _bin(A, True, n, cam, opts, rec, touched, cap)
        assert int(got[3][0]) == 0 and int(got[3][1]) == P, call
        assert torch.equal(want[0][:P], got[0][:P]), call   # sorted record indices
        assert torch.equal(want[1][:P], got[1][:P]), call   # sorted (tile, depth) keys
        assert torch.equal(want[2], got[2]), call           # tile ranges
        assert torch.equal(want[3], got[3]), call           # status word


def test_noalloc_rejects_capacity_beyond_its_static_scratch():
    from paper_2403_16095_b300 import _abi as A
    cam = synth.Camera(64, 48, 50.0, 50.0, 32.0, 24.0)
    opts = A.gs_opts(16, A.GS_MODE_POSE, 1.3, 0.0)
    rec, touched, _ = _records(10, cam, 16, 3)
    cap = A.GS_NOALLOC_MAX_PAIRS + 1
    values = torch.empty(cap, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * 12, dtype=torch.int32, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(A.GsError) as e:
        A.gs_bin_tiles_noalloc(10, [cam], opts, rec, touched, values, None, ranges, status)
    assert e.value.status == A.GS_ERR_INVALID_ARG and "capacity" in str(e.value)
