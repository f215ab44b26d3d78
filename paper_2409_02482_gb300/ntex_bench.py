"""Times one neural texture's forward (network -> grounded texels) and
adjoint (texel gradients -> parameter gradients) on the GPU:

    python -m paper_2409_02482_gb300.ntex_bench [--out-ch 27] [--size 2048] [--fp32]

The network is the fitting benchmark's: a 16-level, 2-feature hash grid of
2^19 rows per level (base resolution 16, growth 1.447) and two 64-wide ReLU
layers, evaluated at the texel centres of a size x size texture, with
random parameters (tables U(+-1e-4), He-normal weights, zero biases) and a
random output gradient.  Prints the best of --repeats CUDA-event timings of
each call (after --warmup untimed rounds) and the workspace status word.
"""

import argparse
import math

import torch

from .render import Context, NeuralTexture


def init_params(nt: NeuralTexture, levels: int, features: int, hidden: int, seed: int = 1) -> None:
    """Random parameters in the vs_ntex_layout order: tables, W0, b0, W1, b1, W2, b2."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    p = torch.zeros(nt.count, dtype=torch.float32)
    off = nt.offsets + [nt.count]
    lf = levels * features
    fan_in = {1: lf, 3: hidden, 5: hidden}
    for i in range(7):
        n = off[i + 1] - off[i]
        if i == 0:
            p[off[0]:off[1]] = (torch.rand(n, generator=g) * 2 - 1) * 1e-4
        elif i in fan_in:
            p[off[i]:off[i + 1]] = torch.randn(n, generator=g) * math.sqrt(2.0 / fan_in[i])
    nt.params.copy_(p)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out-ch", type=int, default=27)
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--fp32", action="store_true", help="FP32 layers instead of the TF32 tensor-core kernels")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--repeats", type=int, default=5)
    a = ap.parse_args(argv)
    ctx = Context(0)
    levels, features, hidden = 16, 2, 64
    nt = NeuralTexture(ctx, levels=levels, features=features, log2_table=19, base_res=16, growth=1.447,
                       hidden=hidden, out_ch=a.out_ch, tex_w=a.size, tex_h=a.size, tensor_cores=not a.fp32)
    init_params(nt, levels, features, hidden)
    pitch = (a.out_ch + 7) // 8 * 8
    tex = torch.zeros((a.size, a.size, pitch), dtype=torch.float16, device="cuda")
    grad = torch.randn((a.size, a.size, pitch), device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    for _ in range(a.warmup):
        nt.forward(tex)
        nt.backward(grad)
    torch.cuda.synchronize()
    fwd, bwd = [], []
    for _ in range(a.repeats):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        nt.forward(tex)
        ev[1].record()
        nt.backward(grad)
        ev[2].record()
        torch.cuda.synchronize()
        fwd.append(ev[0].elapsed_time(ev[1]))
        bwd.append(ev[1].elapsed_time(ev[2]))
    mode = "FP32" if a.fp32 else "TF32"
    print(f"{mode} {a.size}^2 out_ch {a.out_ch}: forward {min(fwd):.3f} ms, adjoint {min(bwd):.3f} ms, "
          f"status {nt.status()}")


if __name__ == "__main__":
    main()
