"""The multi-GPU form of the texture-fitting step, emulated with CPU ranks.

Views are independent, so N GPUs each render and differentiate their own
share of the views and combine the FP32 texel gradients with one all-reduce
sum per fitting step (paper_2409_02482_gb300.shard).  Every box of this
build has one GPU, so the helper's collective is checked here with two gloo
ranks on the CPU: each rank runs the SAME helper the benchmark runs under
torchrun, with the FP64 oracle's adjoint as its gradient callback, and the
all-reduced gradients must equal the single-rank gradient over all views.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2409_02482_gb300.shard import ShardedFittingStep, view_shard

VIEWS = 5


def _setup():
    import synth
    (scene, cams), = synth.config_scene("c2", scale=0.002, views=VIEWS)
    return scene, cams


def _oracle_grads(scene, cams):
    """Gradient callback of a CPU rank: adds the oracle's L2-loss adjoint of
    the given views into the float32 gradient tensors."""
    import oracle

    def compute(grads, views):
        for v in views:
            cam = cams[v]
            rgba, hits, _ = oracle.render(scene, cam, threads=1)
            target = np.random.default_rng(100 + v).random((cam.height, cam.width, 3))
            _, dL = oracle.l2_loss_grad(rgba, target)
            for acc, g in zip(grads, oracle.backward(scene, cam, hits, dL)):
                acc += torch.from_numpy(g.astype(np.float32))
    return compute


def _run_step(rank, world):
    scene, cams = _setup()
    grads = [torch.full(s.tex.shape, 7.0, dtype=torch.float32) for s in scene.shells]   # zeroed by the step
    compute = _oracle_grads(scene, cams)
    step = ShardedFittingStep(grads, lambda views: compute(grads, views), VIEWS, rank=rank, world=world)
    assert step.views == list(range(rank, VIEWS, world))
    out = step()
    return torch.cat([g.reshape(-1) for g in out]).numpy()


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scene, cams = _setup()
    grads = [torch.full(s.tex.shape, 7.0, dtype=torch.float32) for s in scene.shells]
    compute = _oracle_grads(scene, cams)
    step = ShardedFittingStep(grads, lambda views: compute(grads, views), VIEWS)
    assert (step.rank, step.world) == (rank, world)
    got = torch.cat([g.reshape(-1) for g in step()]).numpy()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), got)
    np.save(os.path.join(out_dir, f"views{rank}.npy"), np.array(step.views))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_view_shard_partitions_the_views():
    for n in (0, 1, 5, 100):
        for world in (1, 2, 3, 8):
            parts = [view_shard(n, r, world) for r in range(world)]
            assert sorted(v for p in parts for v in p) == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        view_shard(4, 2, 2)


@pytest.mark.timeout(600)
def test_allreduced_shard_gradients_equal_single_rank(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    full = _run_step(0, 1)     # one rank, every view, no collective
    assert np.abs(full).max() > 0
    views = sorted(int(v) for r in range(world) for v in np.load(tmp_path / f"views{r}.npy"))
    assert views == list(range(VIEWS))
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        # float32 sums of the same terms in another order
        assert np.allclose(got, full, rtol=1e-5, atol=1e-6 * np.abs(full).max())
