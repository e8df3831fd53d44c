"""Learned non-reflecting boundary: training-data generation, training and evaluation.

Training pairs come from the solver itself.  A batch of periodic D2Q5 domains, three times the
physical region's size in each direction, carries seeded pulses that start inside the physical
region.  Every `record_every` steps `lee_batch_edge_samples` reads, for every border cell of the
physical region, the network input (the normalised 3-cell strip) and the target (the population
that streams in from the cell just outside).  A wave that leaves the region needs at least
2 x (region size) steps to wrap around the periodic box and come back, so for
`steps <= 2 * region` the targets are those of an unbounded domain.

Training runs on the library's own kernels: fused forward + backward on the tensor cores,
deterministic gradient reduction, Adam.  Torch only holds the sample buffers and draws the
minibatch permutation.

Evaluation on an open grid compares, against a light-cone-enlarged FP64 periodic run, the
zero-incoming edge, a sponge frame and the learned edge.  The error measure is the space-time
L2 norm of rho' over the physical region (Sec. 9, eq. "L2 space time norm") relative to the
reference's.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs


def _torch():
    import torch

    return torch


def training_domains(batch: int, region: int, rng):
    """Pulse specs of one batch: 1-3 Gaussians per domain with centres inside the physical
    region, amplitude ~ U[1e-4, 1e-3], width ~ U[region / 32, region / 6] cells."""
    specs = []
    for _ in range(batch):
        k = int(rng.integers(1, 4))
        pulses = [(rng.uniform(region, 2 * region), rng.uniform(region, 2 * region), rng.uniform(1e-4, 1e-3),
                   rng.uniform(region / 32.0, region / 6.0)) for _ in range(k)]
        specs.append(pulses)
    return specs


def _pulse_fields_on_device(pulses, n):
    """Density of the pulses on an n x n periodic grid (minimum-image distances), built on the
    device; zero velocity and temperature perturbations."""
    torch = _torch()
    ax = torch.arange(n, dtype=torch.float64, device="cuda")
    rho = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    for cx, cy, a, w in pulses:
        dx = torch.remainder(ax - cx + n / 2.0, n) - n / 2.0
        dy = torch.remainder(ax - cy + n / 2.0, n) - n / 2.0
        rho += a * torch.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (w * w))
    zeros_u = torch.zeros((2, n * n), dtype=torch.float64, device="cuda")
    zeros_t = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    return rho.reshape(-1), zeros_u, zeros_t


def generate_samples(lee, trajectories: int = 5000, region: int = 256, steps: int = 512, record_every: int = 8,
                     batch: int = 96, tau: float = 0.6, seed: int = 5, min_scale: float = 1e-9, stream=None):
    """Runs `trajectories` seeded pulse runs on 3x enlarged periodic domains (FP32, batched, one
    CUDA graph per run length) and returns device tensors (x[rows][16], t[rows]) of border
    samples.  Strips the pulse has not reached (scale below `min_scale`) are dropped, and the
    rest are kept with probability min(1, (s / s90)^2), s90 the 90th percentile of the record's
    scales, which weights the set towards the strips that carry the wave's energy."""
    torch = _torch()
    assert steps <= 2 * region, "waves would wrap around the enlarged box"
    n = 3 * region
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    R = 4 * region
    xs, ts = [], []
    done = 0
    while done < trajectories:
        count = min(batch, trajectories - done)
        specs = training_domains(count, region, rng)
        with lee.Batch("D2Q5", "f32", [(n, n, tau)] * count, stream=stream) as b:
            for d, pulses in enumerate(specs):
                b.init_fields(d, *_pulse_fields_on_device(pulses, n))
            xb = torch.empty((count * R, 16), device="cuda")
            tb = torch.empty(count * R, device="cuda")
            sb = torch.empty(count * R, device="cuda")
            for t in range(0, steps, record_every):
                b.step(record_every, "graph")
                lee.lee_batch_edge_samples(b.b, region, region, region, region, xb, tb, sb)
                live = sb > min_scale
                if not bool(live.any()):
                    continue
                s90 = torch.quantile(sb[live][: 1 << 20], 0.9)
                keep = live & (torch.rand(sb.shape, device="cuda", generator=gen) < (sb / s90) ** 2)
                xs.append(xb[keep].clone())
                ts.append(tb[keep].clone())
        done += count
    return torch.cat(xs), torch.cat(ts)


def train(lee, x, t, steps: int = 20000, batch_rows: int = 8192, lr: float = 2e-3, lr_final: float = 1e-4,
          seed: int = 0, init=None, stream=None, log_every: int = 1000):
    """Adam on minibatches drawn without replacement; cosine learning-rate decay.  Returns the
    FP32 parameter vector and the loss history [(step, loss)]."""
    torch = _torch()
    p0 = init if init is not None else he_init(seed)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    rows = x.shape[0]
    perm = torch.randperm(rows, device="cuda", generator=g)
    pos = 0
    hist = []
    loss = torch.empty(1, device="cuda")
    with lee.Mlp(p0, stream=stream) as m:
        for it in range(steps):
            if pos + batch_rows > rows:
                perm = torch.randperm(rows, device="cuda", generator=g)
                pos = 0
            idx = perm[pos: pos + batch_rows]
            pos += batch_rows
            xb = x.index_select(0, idx).contiguous()
            tb = t.index_select(0, idx).contiguous()
            m.loss_grad(xb, tb, xb.shape[0], None, loss)
            cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / max(steps - 1, 1)))
            m.adam_step(cur)
            if it % log_every == 0 or it == steps - 1:
                hist.append((it, float(loss.item())))
        params = np.empty(lee.MLP_NPARAM, dtype=np.float32)
        m.get_params(params)
    return params, hist


def he_init(seed: int = 0) -> np.ndarray:
    """He-style initial weights (zero biases; the pad column of W1 zero) as FP32."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0, math.sqrt(2.0 / 15), (64, 16))
    w1[:, 15] = 0.0
    parts = [w1.ravel(), np.zeros(64), rng.normal(0, math.sqrt(2.0 / 64), 64 * 64), np.zeros(64),
             rng.normal(0, math.sqrt(1.0 / 64), 64), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def eval_pulses(n: int, seed: int = 5):
    """1-3 off-centre pulses (amplitude 1e-3, width ~ U[16, 32]) inside an n x n domain."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 4))
    return [(rng.uniform(0.2 * n, 0.8 * n), rng.uniform(0.2 * n, 0.8 * n), 1e-3, rng.uniform(16.0, 32.0))
            for _ in range(k)]


def _rho_region(lee, sv, shape, region, out):
    torch = _torch()
    nx, ny = shape[0], shape[1]
    full = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    sv.moments(full, None, None)
    x0, y0, w, h = region
    out.copy_(full.view(ny, nx)[y0: y0 + h, x0: x0 + w])


def evaluate(lee, params, n: int = 1024, steps: int = 3000, sample_every: int = 30, tau: float = 0.6,
             sponge_width: int = 24, sponge_strength: float = 0.5, seed: int = 5, storage: str = "f32",
             stream=None):
    """Open-edge forms against the light-cone-enlarged FP64 periodic reference.  Returns, per
    form, the relative space-time L2 error of rho' on the physical n x n region, the reflected
    fraction (the same ratio restricted to times after the first wave reached an edge), and
    MLUPS per physical cell (the step loop alone, CUDA events)."""
    torch = _torch()
    pulses = eval_pulses(n, seed)
    samples = list(range(sample_every, steps + 1, sample_every))

    def run(shape, bc, offset, kw, st):
        nx, ny = shape[0], shape[1]
        rho = np.zeros(nx * ny)
        for cx, cy, a, w in pulses:
            rho += inputs.gaussian_pulse((nx, ny, 1), a, w, (cx + offset, cy + offset, 0), periodic=(bc == "periodic"))
        u, th = inputs.zero_rest(2, nx * ny)
        rec = torch.empty((len(samples), n, n), dtype=torch.float64, device="cuda")
        with lee.Solver("D2Q5", (nx, ny, 1), tau, storage=st, bc=bc, stream=stream, **kw) as sv:
            if bc == "open_learned":
                sv.set_boundary_mlp(params)
            sv.init_fields(rho, u, th)
            ms = 0.0
            done = 0
            for k, t in enumerate(samples):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                sv.step(t - done)
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                done = t
                _rho_region(lee, sv, shape, (offset, offset, n, n), rec[k])
        return rec, ms

    margin = steps + 8
    ref, _ = run((n + 2 * margin, n + 2 * margin, 1), "periodic", margin, {}, "f64")
    out = {"workload": f"{n}x{n} open D2Q5, tau={tau}, {len(pulses)} pulses (A=1e-3, w 16-32), {steps} steps, "
                       f"{storage}; reference FP64 periodic {n + 2 * margin}^2 (light cone)",
           "forms": {}}
    # first time a pulse's 3-sigma edge reaches the boundary (lattice speed 1 bound)
    dist = min(min(cx, cy, n - cx, n - cy) - 1.5 * w for cx, cy, a, w in pulses)
    late = torch.tensor([t >= max(dist, 0) for t in samples], device="cuda")
    ref_norm = torch.linalg.norm(ref)
    ref_late = torch.linalg.norm(ref[late])
    forms = [("zero", (n, n, 1), "open_zero", 0, {}),
             ("sponge", (n + 2 * sponge_width, n + 2 * sponge_width, 1), "open_sponge", sponge_width,
              {"sponge_width": sponge_width, "sponge_strength": sponge_strength}),
             ("learned", (n, n, 1), "open_learned", 0, {})]
    for name, shape, bc, off, kw in forms:
        rec, ms = run(shape, bc, off, kw, storage)
        err = float(torch.linalg.norm(rec - ref) / ref_norm)
        refl = float(torch.linalg.norm((rec - ref)[late]) / ref_late)
        out["forms"][name] = {"grid": list(shape[:2]), "rel_l2_spacetime": err, "reflected_fraction": refl,
                              "mlups_physical": round(n * n * steps / (ms / 1e3) / 1e6, 1), "ms": round(ms, 2)}
    return out


def main(argv=None):
    import argparse
    import json

    import paper_1601_08103_gb300 as lee

    ap = argparse.ArgumentParser(description="train and evaluate the learned boundary")
    ap.add_argument("--trajectories", type=int, default=5000)
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--eval-n", type=int, default=1024)
    ap.add_argument("--eval-steps", type=int, default=3000)
    ap.add_argument("--out", default=None, help="write the trained FP32 parameters here (.npy)")
    args = ap.parse_args(argv)
    lee.load()
    t0 = time.time()
    x, t = generate_samples(lee, trajectories=args.trajectories)
    t1 = time.time()
    params, hist = train(lee, x, t, steps=args.train_steps)
    t2 = time.time()
    if args.out:
        np.save(args.out, params)
    ev = evaluate(lee, params, n=args.eval_n, steps=args.eval_steps)
    ev["training"] = {"samples": int(x.shape[0]), "trajectories": args.trajectories, "gen_s": round(t1 - t0, 1),
                      "train_s": round(t2 - t1, 1), "loss_history": hist}
    print(json.dumps(ev))


if __name__ == "__main__":
    main()
