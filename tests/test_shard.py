"""Frame sharding across ranks, on CPU with gloo (world size 2).

Each rank takes its frames of a 4-keyframe window, computes their gradients
(the FP64 oracle stands in for the per-rank GPU backward, which needs no
collective) and sums the per-Gaussian gradients with one all-reduce. The
result must equal the single-process sum over all frames."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2403_16095_b300.shard import allreduce_gaussian_grads, frames_for_rank

PARAMS = ("means", "log_scales", "quats", "opacity_logit", "colors", "nu")


def _window():
    sc, cam, T = synth.tiny_scene()
    Ts = [np.asarray(T, np.float64)]
    for k in range(1, 4):
        Ts.append(synth.jitter_pose(Ts[0], 1200 + k, trans=0.05, rot_deg=3.0))
    tgt = [synth.random_targets(cam, 1200 + 10 + f) for f in range(4)]
    return sc, cam, Ts, tgt


def _frame_grads(sc, cam, Ts, tgt, frames):
    out = {k: np.zeros_like(np.asarray(getattr(sc, k), np.float64)) for k in PARAMS}
    poses = {}
    for f in frames:
        og = oracle.grad(sc, cam, Ts[f], oracle.LossSpec(0.7, 0.25, 0.1, 0.1, 0.025, tgt[f][0][0], tgt[f][1][0]))
        for k in PARAMS:
            out[k] += og[k]
        poses[f] = og["pose"]
    return out, poses


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, cam, Ts, tgt = _window()
        mine = frames_for_rank(len(Ts), rank, world)
        g, poses = _frame_grads(sc, cam, Ts, tgt, mine)
        t = {k: torch.from_numpy(v.copy()) for k, v in g.items()}
        allreduce_gaussian_grads(t)
        q.put((rank, mine, {k: v.numpy() for k, v in t.items()}, poses))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_frames_for_rank_partitions_the_window():
    for n in (0, 1, 4, 7, 16):
        for w in (1, 2, 3, 8):
            got = sorted(f for r in range(w) for f in frames_for_rank(n, r, w))
            assert got == list(range(n))
            sizes = [len(frames_for_rank(n, r, w)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        frames_for_rank(4, 2, 2)


def test_single_process_allreduce_is_identity():
    t = {"a": torch.arange(6.0)}
    assert allreduce_gaussian_grads(t)["a"].tolist() == list(range(6))


def test_two_rank_frame_sharded_sum_equals_single_process_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc, cam, Ts, tgt = _window()
    want, want_pose = _frame_grads(sc, cam, Ts, tgt, range(len(Ts)))
    owners = {}
    for rank, frames, g, poses in res:
        for f in frames:
            owners[f] = rank
            assert np.array_equal(poses[f], want_pose[f])
        for k in PARAMS:
            scale = np.abs(want[k]).max()
            assert np.abs(g[k] - want[k]).max() <= 1e-12 * max(scale, 1e-300), k
    assert sorted(owners) == list(range(len(Ts)))
    # both ranks hold the same summed gradients
    a, b = res[0][2], res[1][2]
    for k in PARAMS:
        assert np.array_equal(a[k], b[k])


def test_window_slice_of_uneven_frames():
    """A rank's share of a window of frames of different sizes: its cameras,
    poses and the planar per-frame RGB-D targets, cut at each frame's pixel
    offset, in the rank's frame order."""
    from paper_2403_16095_b300.shard import window_slice
    cams = [synth.Camera(w, h, 50.0, 50.0, w / 2, h / 2) for w, h in ((4, 3), (5, 2), (2, 2), (3, 3))]
    sizes = [c.width * c.height for c in cams]
    T = torch.arange(4 * 12, dtype=torch.float32).reshape(4, 3, 4)
    tc = torch.cat([torch.full((3 * n,), float(f)) for f, n in enumerate(sizes)])
    td = torch.cat([torch.full((n,), 10.0 + f) for f, n in enumerate(sizes)])
    for frames in ([1, 3], [0, 2], [3], []):
        c, Tr, tcr, tdr = window_slice(cams, T, tc, td, frames)
        assert [x.width for x in c] == [cams[f].width for f in frames]
        assert torch.equal(Tr, T[frames].reshape(-1) if frames else T[:0].reshape(-1))
        assert torch.equal(tcr, torch.cat([torch.full((3 * sizes[f],), float(f)) for f in frames])
                           if frames else tc[:0])
        assert torch.equal(tdr, torch.cat([torch.full((sizes[f],), 10.0 + f) for f in frames]) if frames else td[:0])


def test_rank_without_frames_contributes_zeros():
    """With more ranks than keyframes, a rank that owns no frame builds no
    rasterizer and its step writes zero gradients (then joins the all-reduce,
    the identity in a single process)."""
    from paper_2403_16095_b300.shard import ShardedWindow
    cams = [synth.Camera(8, 6, 10.0, 10.0, 4.0, 3.0)] * 3
    T = torch.zeros(3, 3, 4)
    sw = ShardedWindow(cams, 5, T, torch.zeros(3 * 3 * 48), torch.zeros(3 * 48), rank=4, world=6)
    assert sw.frames == [] and sw.rast is None and sw.pose_grads() == {} and sw.status() == (0, 0)
    grads = {k: torch.ones(5, 3) for k in PARAMS}
    sw.step(None, grads)
    assert all(float(v.abs().sum()) == 0.0 for v in grads.values())
