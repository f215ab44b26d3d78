"""The multi-GPU form of the texture-fitting step, emulated with CPU ranks.

Views are independent, so N GPUs would each render and differentiate their
own share of the views and combine the FP32 texel gradients with one
all-reduce sum per fitting step.  Every box of this build has one GPU, so the
benchmark runs replicas; the reduction itself is checked here with two gloo
ranks on the CPU, using the FP64 oracle's adjoint as each rank's work: the
all-reduced partial gradients must equal the single-rank gradient over all
views.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

VIEWS = 4


def _shard_gradient(rank, world):
    import oracle
    import synth
    (scene, cams), = synth.config_scene("c2", scale=0.002, views=VIEWS)
    grads = [np.zeros(s.tex.shape, np.float64) for s in scene.shells]
    for v in range(rank, VIEWS, world):
        cam = cams[v]
        rgba, hits, _ = oracle.render(scene, cam, threads=1)
        target = np.random.default_rng(100 + v).random((cam.height, cam.width, 3))
        _, dL = oracle.l2_loss_grad(rgba, target)
        for acc, g in zip(grads, oracle.backward(scene, cam, hits, dL)):
            acc += g
    return np.concatenate([g.reshape(-1) for g in grads])


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = torch.from_numpy(_shard_gradient(rank, world))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.timeout(600)
def test_allreduced_shard_gradients_equal_single_rank(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    full = _shard_gradient(0, 1)
    assert np.abs(full).max() > 0
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert np.allclose(got, full, rtol=1e-12, atol=1e-15 * np.abs(full).max())
