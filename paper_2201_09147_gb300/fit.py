"""Offline bootstrap fitter for the nested SIREN sequences (input generator).

Produces the trained sine MLPs that the multiscale tracer consumes.  The
paper trains its networks with an external framework it only cites (Sec. 2,
Sec. 3.3); this stand-in fits each network of a sequence independently to the
seeded analytic scene of ``inputs.sphere_scene`` with plain PyTorch autograd:

    loss = mean |f(x) - g(x)|                         (SDF values)
         + lam_n * mean (1 - cos(grad f(x), grad g(x)))  (normals, near surface)
         + lam_e * mean | |grad f(x)| - 1 |              (Eikonal)

on a batch that is half near-surface (sphere-surface points plus N(0, 0.02)
jitter) and half uniform in [-1, 1]^3.  Networks are stored unfolded (SIREN
parametrisation, omega0 = omega = 30) in SDFN files.

The thresholds of the sequence then follow Prop. 2 (Sec. 3.3) with the
infinity norm estimated as the maximum over sampled points, as the paper
prescribes; that estimate lives in the tests (it needs the oracle).

This module is not on the rendering path: nothing in the CUDA library or its
binding imports it.  With ``--native`` the same objective and Adam run on the
GPU through the library's training kernels instead of torch autograd.  Usage:

    python -m paper_2201_09147_gb300.fit --out paper_2201_09147_gb300/scenes [--native]
"""
from __future__ import annotations

import argparse
import json
import math
import time
from pathlib import Path

import numpy as np
import torch

from . import inputs

SCENES_DIR = Path(__file__).resolve().parent / "scenes"

# name -> (width, n_hidden, steps[, in_dim]); 4-D nets take (x, y, z, t) of the animated scene
SEQUENCE_NETS = {
    "a8_64x1_t": (64, 1, 3000, 4),
    "a8_256x3_t": (256, 3, 3000, 4),
    "s8_64x1": (64, 1, 3000),
    "s8_64x2": (64, 2, 3000),
    "s8_128x2": (128, 2, 3000),
    "s8_256x1": (256, 1, 3000),
    "s8_256x2": (256, 2, 3000),
    "s8_256x3": (256, 3, 3000),
    "a8_128x2_t": (128, 2, 3000, 4),
}
# the nested sequence of the 3-level workload (and the 4-D middle network of the animated pair)
# is fitted natively, on the GPU, with BF16 tensor-core training: 4000 steps of 2^18 points
NATIVE_NETS = {"s8_64x2", "s8_128x2", "s8_256x2", "a8_128x2_t"}
NATIVE_STEPS, NATIVE_BATCH = 4000, 1 << 18


class Siren(torch.nn.Module):
    def __init__(self, net: inputs.SineNet):
        super().__init__()
        self.omega0, self.omega = net.omega0, net.omega
        self.layers = torch.nn.ModuleList()
        for w, b in zip(net.weights, net.biases):
            lin = torch.nn.Linear(w.shape[1], w.shape[0])
            with torch.no_grad():
                lin.weight.copy_(torch.from_numpy(np.asarray(w, np.float32)))
                lin.bias.copy_(torch.from_numpy(np.asarray(b, np.float32)))
            self.layers.append(lin)

    def forward(self, x):
        n = len(self.layers)
        for i, lin in enumerate(self.layers):
            x = lin(x)
            if i < n - 1:
                x = torch.sin((self.omega0 if i == 0 else self.omega) * x)
        return x[..., 0]

    def to_sinenet(self, template: inputs.SineNet) -> inputs.SineNet:
        ws = [lin.weight.detach().cpu().numpy().astype(np.float32) for lin in self.layers]
        bs = [lin.bias.detach().cpu().numpy().astype(np.float32) for lin in self.layers]
        return inputs.SineNet(template.in_dim, template.width, template.n_hidden, template.omega0,
                              template.omega, ws, bs, folded=False)


def scene_torch(scene: inputs.SphereScene, p: torch.Tensor, centres=None):
    """Analytic scene value and gradient (torch, float32); `centres` (n, m, 3) overrides per point."""
    c = torch.as_tensor(scene.centres, dtype=p.dtype, device=p.device) if centres is None else centres
    r = torch.as_tensor(scene.radii, dtype=p.dtype, device=p.device)
    diff = p[:, None, :] - (c[None] if c.dim() == 2 else c)
    dist = diff.norm(dim=-1)
    d = dist - r[None]
    dmin, arg = d.min(dim=1)
    nrm = diff[torch.arange(p.shape[0]), arg] / dist[torch.arange(p.shape[0]), arg, None].clamp_min(1e-12)
    a, fr = scene.amp, scene.freq
    sx, sy, sz = torch.sin(fr * p[:, 0]), torch.sin(fr * p[:, 1]), torch.sin(fr * p[:, 2])
    cx, cy, cz = torch.cos(fr * p[:, 0]), torch.cos(fr * p[:, 1]), torch.cos(fr * p[:, 2])
    val = dmin + a * sx * sy * sz
    grad = nrm + a * fr * torch.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz], dim=1)
    return val, grad


def sample_batch(scene: inputs.SphereScene, gen: torch.Generator, n: int):
    half = n // 2
    k = torch.randint(0, len(scene.radii), (half,), generator=gen)
    u = torch.randn(half, 3, generator=gen)
    u = u / u.norm(dim=1, keepdim=True)
    c = torch.as_tensor(scene.centres, dtype=torch.float32)[k]
    r = torch.as_tensor(scene.radii, dtype=torch.float32)[k]
    near = c + r[:, None] * u + 0.02 * torch.randn(half, 3, generator=gen)
    near = near.clamp(-1.0, 1.0)
    unif = torch.rand(n - half, 3, generator=gen) * 2.0 - 1.0
    return torch.cat([near, unif], dim=0), half


def animated_centres(seed: int, t: torch.Tensor):
    """Centres of inputs.sphere_scene(seed, time=t) for a batch of times, (n, m, 3)."""
    s0 = inputs.sphere_scene(seed)
    s1 = inputs.sphere_scene(seed, time=0.0)
    # the phases are drawn after the centres and radii: recover them from time 0
    delta0 = (s1.centres - s0.centres) / 0.15
    phase = torch.as_tensor(np.arctan2(delta0[:, 1], delta0[:, 0]), dtype=torch.float32)
    c0 = torch.as_tensor(s0.centres, dtype=torch.float32)
    ang = 2.0 * math.pi * t[:, None] + phase[None, :]
    off = 0.15 * torch.stack([torch.cos(ang), torch.sin(ang), torch.zeros_like(ang)], dim=-1)
    return c0[None] + off


def fit_net(scene, width, n_hidden, steps, seed=0, batch=1 << 14, lr=1e-4, lam_n=0.1, lam_e=0.05,
            device="cpu", log_every=500, in_dim=3, scene_seed=1):
    torch.manual_seed(seed)
    gen = torch.Generator().manual_seed(seed)
    template = inputs.siren_init(seed, width, n_hidden, in_dim=in_dim)
    model = Siren(template).to(device)
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=steps, eta_min=lr * 0.05)
    t0 = time.time()
    for it in range(steps):
        x, half = sample_batch(scene, gen, batch)
        centres = None
        if in_dim == 4:
            # time in [0, 1); near-surface samples follow the moving spheres
            tt = torch.rand(batch, generator=gen)
            centres = animated_centres(scene_seed, tt)
            k = torch.randint(0, len(scene.radii), (half,), generator=gen)
            shift = centres[torch.arange(half), k] - torch.as_tensor(scene.centres, dtype=torch.float32)[k]
            x = torch.cat([(x[:half] + shift).clamp(-1.0, 1.0), x[half:]], dim=0)
        x = x.to(device).requires_grad_(True)
        gv, gg = scene_torch(scene, x.detach(), centres)
        inp = torch.cat([x, tt[:, None].to(device)], dim=1) if in_dim == 4 else x
        f = model(inp)
        (df,) = torch.autograd.grad(f.sum(), x, create_graph=True)
        l_val = (f - gv).abs().mean()
        cos = torch.nn.functional.cosine_similarity(df[:half], gg[:half], dim=1)
        l_n = (1.0 - cos).mean()
        l_e = (df.norm(dim=1) - 1.0).abs().mean()
        loss = l_val + lam_n * l_n + lam_e * l_e
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if log_every and (it % log_every == 0 or it == steps - 1):
            print(f"  ({width},{n_hidden}) in{in_dim} it {it:5d} loss {loss.item():.5f} val {l_val.item():.5f} "
                  f"n {l_n.item():.4f} eik {l_e.item():.4f}  {time.time() - t0:.0f}s", flush=True)
    return model.cpu().to_sinenet(template)


def fit_net_native(scene, width, n_hidden, steps, seed=0, batch=1 << 18, lr=1e-4, lam_n=0.1, lam_e=0.05,
                   log_every=500, scene_seed=1, in_dim=3, precision=None):
    """The same objective and Adam, run natively on the GPU through the library's
    training kernels (sdf_train_forward / sdf_fit_loss / sdf_train_backward /
    sdf_adam_step), parameters in folded form; by default with BF16 tensor-core
    contractions.  The batches (half near the surface with N(0, 0.02) jitter,
    half uniform; 4-D: a uniform time per point, the near-surface half following
    the moving spheres) are drawn on the GPU by torch from a generator seeded
    with `seed`, the targets from the analytic scene."""
    from . import sdfnn
    precision = sdfnn.SDF_BF16 if precision is None else precision
    dev = torch.device("cuda")
    template = inputs.siren_init(seed, width, n_hidden, in_dim=in_dim)
    shape, theta = sdfnn.theta_from_sdfn(inputs.net_to_bytes(template))
    th = torch.from_numpy(theta).to(dev)
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    gen = torch.Generator(device=dev).manual_seed(seed)
    c_all = torch.as_tensor(scene.centres, dtype=torch.float32, device=dev)
    r_all = torch.as_tensor(scene.radii, dtype=torch.float32, device=dev)
    half = batch // 2
    near = torch.zeros(batch, dtype=torch.uint8, device=dev)
    near[:half] = 1
    ws = None
    t0 = time.time()
    for it in range(steps):
        k = torch.randint(0, len(scene.radii), (half,), generator=gen, device=dev)
        u = torch.randn(half, 3, generator=gen, device=dev)
        u = u / u.norm(dim=1, keepdim=True)
        jit = 0.02 * torch.randn(half, 3, generator=gen, device=dev)
        unif = torch.rand(batch - half, 3, generator=gen, device=dev) * 2.0 - 1.0
        tt, centres = None, None
        if in_dim == 4:
            tt = torch.rand(batch, generator=gen, device=dev)
            centres = animated_centres(scene_seed, tt.cpu()).to(dev)
            cnear = centres[torch.arange(half, device=dev), k]
        else:
            cnear = c_all[k]
        x = torch.cat([(cnear + r_all[k][:, None] * u + jit).clamp(-1.0, 1.0), unif], dim=0)
        gv, gg = scene_torch(scene, x, centres)
        # cosine schedule to lr / 20, as the torch fitter
        lr_t = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * it / steps)))
        # the parameters are trained folded (W' = omega W): Adam's steps on the sine layers are
        # scaled by omega so that they match the torch fitter's steps on the SIREN parameters
        loss, ws = sdfnn.fit_step(shape, th, m, v, it + 1, x.T.contiguous(), gv.contiguous(), gg.T.contiguous(), near,
                                  lam_n=lam_n, lam_e=lam_e, lr=lr_t, workspace=ws, precision=precision,
                                  pt_time=tt, sine_lr_scale=template.omega)
        if log_every and (it % log_every == 0 or it == steps - 1):
            lv = loss.cpu().numpy()
            print(f"  ({width},{n_hidden}) in{in_dim} native it {it:5d} loss {lv[3]:.5f} val {lv[0]:.5f} "
                  f"n {lv[1]:.4f} eik {lv[2]:.4f}  {time.time() - t0:.0f}s", flush=True)
    sdfnn.sync_status()
    return inputs.net_from_bytes(sdfnn.sdfn_from_theta(shape, th.cpu().numpy()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=str(SCENES_DIR))
    ap.add_argument("--nets", default=",".join(SEQUENCE_NETS))
    ap.add_argument("--steps", type=int, default=0, help="override the step count")
    ap.add_argument("--device", default="cpu")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--native", action="store_true",
                    help="fit every listed network on the GPU with the library's BF16 training kernels")
    args = ap.parse_args()
    if args.threads:
        torch.set_num_threads(args.threads)
    out = Path(args.out)
    out.mkdir(parents=True, exist_ok=True)
    scene = inputs.sphere_scene(seed=1)
    meta_path = out / "fit_meta.json"
    meta = json.loads(meta_path.read_text()) if meta_path.exists() else {}
    for name in args.nets.split(","):
        w, k, steps, *rest = SEQUENCE_NETS[name]
        in_dim = rest[0] if rest else 3
        native = args.native or name in NATIVE_NETS
        steps = args.steps or (NATIVE_STEPS if native else steps)
        print(f"fitting {name}: ({w},{k}) in_dim {in_dim}, {steps} steps", flush=True)
        if native:
            net = fit_net_native(scene, w, k, steps, batch=NATIVE_BATCH, in_dim=in_dim)
            info = {"fitter": "native (library training kernels, BF16 tensor cores)", "batch": NATIVE_BATCH}
        else:
            net = fit_net(scene, w, k, steps, device=args.device, in_dim=in_dim)
            info = {"fitter": "torch (bootstrap)", "batch": 1 << 14}
        inputs.write_net(out / f"{name}.sdfn", net)
        meta[name] = {"width": w, "n_hidden": k, "in_dim": in_dim, "steps": steps, "seed": 0, "scene_seed": 1,
                      **info}
    meta_path.write_text(json.dumps(meta, indent=1, sort_keys=True) + "\n")


if __name__ == "__main__":
    main()
