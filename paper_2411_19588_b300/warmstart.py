"""Learned warm-start of the medium, next to the plain fit (Sec. IV-C).

The paper fits all Gaussian and medium parameters with Adam from a fixed
initial medium. This form renders many generated scenes with known water
(beta_D, beta_B ~ U[0.05, 0.6] /m, B_inf ~ U[0.05, 0.4] per channel), turns
each view into one feature row (``mlp.featurise``), trains the BF16 MLP on
them, and at fit time initialises the medium from the network's prediction
for a few target views. The plain fit stays the fallback and the judge: the
warm fit counts iterations and wall time until it reaches the PSNR the plain
fit ends at.

Every render, feature, GEMM and update runs in libsplash; this module only
drives the loop (scene generation uses torch's RNG on the device).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import backscatter as BSC
from . import mlp as M
from . import render as R
from . import scenes
from . import schedule as SCH

DEFAULT_MEDIUM = [0.1] * 9
# MCMC densification (the cited method's schedule: relocation every 100
# iterations from 500 to 25,000, dead below opacity 0.005, noise weight 5e5)
MCMC_DEFAULTS = {"start": 500, "stop": 25_000, "every": 100, "min_opacity": 0.005, "lambda_noise": 5e5}
# learning rates of the fit (3DGS values the paper keeps, appendix "Experimental Setup")
FIT_LR = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 5e-2, "sh": 2.5e-3, "medium": 2.5e-3}


def random_media(gen: torch.Generator, k: int, device="cuda") -> torch.Tensor:
    """[k, 9]: beta_D, beta_B ~ U[0.05, 0.6], B_inf ~ U[0.05, 0.4]."""
    u = torch.rand((k, 9), generator=gen, device=device)
    lo = torch.tensor([0.05] * 9, device=device)
    hi = torch.tensor([0.6] * 6 + [0.4] * 3, device=device)
    return (lo + (hi - lo) * u).contiguous()


def jitter_camera(rng: np.random.Generator, z_mid: float, width: int, height: int, fx: float) -> scenes.Camera:
    eye = rng.normal(0.0, 0.15, 3)
    target = np.array([rng.normal(0.0, 0.2), rng.normal(0.0, 0.2), z_mid])
    return scenes.look_at(eye, target, width, height, fx, fx)


def generate(renderer: R.Renderer, n_scenes: int, views_per_scene: int, n_gauss: int = 300_000, width: int = 1280,
             height: int = 854, fx: float = 1200.0, seed: int = 5, z_near=(1.0, 3.0), z_far=(7.0, 15.0)):
    """Feature bank [n, ROW] (BF16) and medium targets [n, 9] from
    n_scenes x views_per_scene renders of generated patch scenes (depth range
    drawn per scene so that it covers both the 1-8 m and 2-15 m families)."""
    n = n_scenes * views_per_scene
    bank = torch.empty((n, M.ROW), dtype=torch.bfloat16, device="cuda")
    targets = torch.empty((n, M.OUT), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    st = renderer.state()
    image = torch.empty((3, height, width), device="cuda")
    depth = torch.empty((height, width), device="cuda")
    depth01 = torch.empty((height, width), device="cuda")
    i = 0
    for s in range(n_scenes):
        z0, z1 = rng.uniform(*z_near), rng.uniform(*z_far)
        params = scenes.patch_scene_device(n_gauss, seed * 100_003 + s, (z0, z1), width, height, fx)
        media = random_media(gen, views_per_scene)
        targets[i:i + views_per_scene] = media
        for v in range(views_per_scene):
            cam = jitter_camera(rng, 0.5 * (z0 + z1), width, height, fx)
            renderer.forward(st, params, media[v], cam, image, depth, depth01)
            M.featurise(renderer, image, depth, cam.z_far, bank[i])
            i += 1
    return bank, targets


def train(net: M.Mlp, bank: torch.Tensor, targets: torch.Tensor, epochs: int = 30, batch: int = 256, lr: float = 1e-3,
          val_frac: float = 0.1, seed: int = 0) -> dict:
    """Adam with a cosine learning-rate decay; returns train/validation
    losses (mean |log p - log t|) and the wall time."""
    n = bank.shape[0]
    gen = torch.Generator(device="cuda").manual_seed(seed)
    perm = torch.randperm(n, generator=gen, device="cuda").to(torch.int32)
    n_val = max(1, int(round(n * val_frac)))
    val, tr = perm[:n_val].contiguous(), perm[n_val:].contiguous()
    steps_per_epoch = max(1, (tr.numel() + batch - 1) // batch)
    total = epochs * steps_per_epoch
    loss_sum = torch.zeros(1, device="cuda")
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 0
    for ep in range(epochs):
        order = tr[torch.randperm(tr.numel(), generator=gen, device="cuda")]
        loss_sum.zero_()
        for b in range(steps_per_epoch):
            idx = order[b * batch:(b + 1) * batch].contiguous()
            step_lr = lr * 0.5 * (1 + math.cos(math.pi * k / total))
            loss_sum += net.step(bank, targets, idx=idx, lr=step_lr)
            k += 1
        hist.append(loss_sum.item() / steps_per_epoch)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"train_loss": hist, "val_loss": evaluate(net, bank, targets, val), "wall_s": wall, "steps": k,
            "n_train": int(tr.numel()), "n_val": n_val}


def evaluate(net: M.Mlp, bank: torch.Tensor, targets: torch.Tensor, idx: torch.Tensor) -> float:
    """Mean |log p - log t| over the rows idx (the network's own loss kernel)."""
    tot, cnt = 0.0, 0
    for b in range(0, idx.numel(), net.max_batch):
        chunk = idx[b:b + net.max_batch].contiguous()
        tot += net.step(bank, targets, idx=chunk, lr=None).item() * chunk.numel()
        cnt += chunk.numel()
    return tot / cnt


def log_error(pred, truth) -> float:
    """Mean |log p - log t| of two 9-vectors."""
    p, t = np.asarray(pred, np.float64), np.asarray(truth, np.float64)
    return float(np.abs(np.log(p) - np.log(t)).mean())


class Fit:
    """The plain fit: forward, L1 + lam (1 - SSIM), fused backward + Adam on
    every Gaussian and medium parameter (medium clamped at 0), one view per
    iteration in a fixed shuffled order. With lambda_est > 0 the loss also
    carries Eq. 9's lambda_est L_best term: every estimate_every iterations
    (and at the first) the backscatter estimate (Alg. 1/2) is recomputed
    from the iteration's target image and the depth just rendered at that
    view, and the prior's gradient joins the medium step. With schedule=True
    the appendix's schedule applies: the position learning rate decays
    (schedule.position_lr) and the opacities are reset every
    reset_every iterations. With densify (a dict: start, stop, every,
    grad_threshold, min_opacity, percent_dense; defaults from
    schedule.DENSIFY) the fit gathers the densification statistics while the
    (1-based) iteration is below stop and densifies at every multiple of
    `every` above start. With mcmc (a dict: start, stop, every, min_opacity,
    lambda_noise; defaults MCMC_DEFAULTS) the fit densifies the way Sec. IV-D
    adopts instead: after every Adam step the position noise, and at every
    multiple of `every` in [start, stop) a relocation of the dead Gaussians
    (the count stays fixed)."""

    def __init__(self, renderer: R.Renderer, params: dict, medium, cams, targets, lam: float = 0.2, lr=None,
                 lambda_est: float = 0.0, estimate_every: int = 500, schedule: bool = False,
                 reset_every: int = SCH.OPACITY_RESET_EVERY, densify: dict | None = None, seed: int = 0,
                 pixel: bool = False, mcmc: dict | None = None):
        self.r = renderer
        self.params = {k: (v.clone() if isinstance(v, torch.Tensor) else v) for k, v in params.items()}
        self.medium = torch.as_tensor(np.asarray(medium, np.float32)).cuda().contiguous()
        self.cams, self.targets, self.lam = cams, targets, lam
        self.lr = dict(FIT_LR if lr is None else lr)
        names = R.PARAM_NAMES + ("medium",)
        tens = dict(self.params)
        tens["medium"] = self.medium
        self.m = {k: torch.zeros_like(tens[k]) for k in names}
        self.v = {k: torch.zeros_like(tens[k]) for k in names}
        self.st = renderer.state()
        H, W = cams[0].height, cams[0].width
        self.image = torch.empty((3, H, W), device="cuda")
        self.depth = torch.empty((H, W), device="cuda")
        self.depth01 = torch.empty((H, W), device="cuda")
        self.it = 0
        self.order = np.random.default_rng(0).permutation(len(cams))
        self.lambda_est, self.estimate_every = float(lambda_est), int(estimate_every)
        self.estimate = BSC.new_result() if self.lambda_est > 0 else None
        self.estimates_done = 0
        self.schedule, self.reset_every, self.resets_done = bool(schedule), int(reset_every), 0
        self.pixel = bool(pixel)  # Eq. 5 per pixel instead of per Gaussian and water segment
        self.densify = None if densify is None else {**SCH.DENSIFY, **densify}
        self.densify_steps, self.counts = 0, [self.params["means"].shape[0]]
        self.stats = None
        if densify is not None and mcmc is not None:
            raise ValueError("densify and mcmc are alternatives")
        self.mcmc = None if mcmc is None else {**MCMC_DEFAULTS, **mcmc}
        self.relocations, self.dead_relocated = 0, []
        if self.mcmc is not None:
            self.gen = torch.Generator(device="cuda").manual_seed(seed)
        if self.densify is not None:
            self.stats = torch.zeros((self.params["means"].shape[0], 2), device="cuda")
            centres = np.stack([-c.world_to_cam[:, :3].T @ c.world_to_cam[:, 3] for c in cams])
            self.extent = 1.1 * float(np.linalg.norm(centres - centres.mean(0), axis=1).max())
            self.gen = torch.Generator(device="cuda").manual_seed(seed)

    def step(self):
        if self.schedule:
            self.lr["means"] = SCH.position_lr(self.it)
            if self.it > 0 and self.it % self.reset_every == 0:
                R.opacity_reset(self.params["opacity_logits"], self.m["opacity_logits"], self.v["opacity_logits"],
                                SCH.OPACITY_RESET_VALUE)
                self.resets_done += 1
        k = int(self.order[self.it % len(self.cams)])
        cam = self.cams[k]
        self.r.forward(self.st, self.params, self.medium, cam, self.image, self.depth, self.depth01, pixel=self.pixel)
        prior = None
        if self.estimate is not None:
            if self.it % self.estimate_every == 0:
                BSC.estimate(self.r, self.targets[k], self.depth, result=self.estimate)
                self.estimates_done += 1
            prior = BSC.prior_of(self.estimate)
        loss, gimg = self.r.loss(self.st, self.image, self.targets[k], self.lam)
        self.it += 1
        d = self.densify
        gather = d is not None and self.it < d["stop"]  # 1-based iteration, as in 3DGS
        self.r.backward_adam(self.st, self.params, self.medium, cam, gimg, self.m, self.v, self.lr, self.it,
                             prior=prior, lambda_est=self.lambda_est, densify_stats=self.stats if gather else None,
                             pixel=self.pixel)
        if gather and self.it > d["start"] and self.it % d["every"] == 0:
            self._densify()
        mc = self.mcmc
        if mc is not None:
            n = self.params["means"].shape[0]
            eta = torch.randn((n, 3), generator=self.gen, device="cuda")
            R.mcmc_noise(self.params, eta, self.lr["means"], mc["lambda_noise"])
            if mc["start"] <= self.it < mc["stop"] and self.it % mc["every"] == 0:
                u = torch.rand(n, generator=self.gen, device="cuda")
                self.dead_relocated.append(R.mcmc_relocate(self.r, self.params, self.m, self.v, u, mc["min_opacity"]))
                self.relocations += 1
        return loss

    def _densify(self):
        d = self.densify
        n = self.params["means"].shape[0]
        noise = torch.randn((n, 2, 3), generator=self.gen, device="cuda")
        p, m, v = R.densify(self.r, self.params, self.m, self.v, self.stats, noise, self.extent, d["grad_threshold"],
                            d["min_opacity"], d["percent_dense"])
        self.params, self.m, self.v = p, m, v
        self.stats = torch.zeros((p["means"].shape[0], 2), device="cuda")
        self.densify_steps += 1
        self.counts.append(p["means"].shape[0])

    def psnr(self, views) -> float:
        """Mean PSNR (images clipped to [0, 1]) over the given views."""
        vals = []
        for k in views:
            self.r.forward(self.st, self.params, self.medium, self.cams[k], self.image, self.depth, self.depth01,
                           pixel=self.pixel)
            mse = torch.mean((self.image.clamp(0, 1) - self.targets[k].clamp(0, 1)) ** 2)
            vals.append(mse)
        mse = torch.stack(vals)
        return float((-10.0 * torch.log10(mse)).mean())


def predict_medium(renderer: R.Renderer, net: M.Mlp, params: dict, cams, targets, views) -> np.ndarray:
    """Medium predicted from target views: each view's feature row pairs the
    target image with the depth of the current scene render at that view; the
    per-view predictions are averaged in log space."""
    st = renderer.state()
    rows = torch.empty((len(views), M.ROW), dtype=torch.bfloat16, device="cuda")
    med0 = torch.tensor(DEFAULT_MEDIUM, dtype=torch.float32, device="cuda")
    for j, k in enumerate(views):
        _, depth, _ = renderer.forward(st, params, med0, cams[k])
        M.featurise(renderer, targets[k], depth, cams[k].z_far, rows[j])
    pred = net.predict(rows).double().cpu().numpy()
    return np.exp(np.log(pred).mean(0))


def fit_curve(fit: Fit, iters: int, eval_every: int, eval_views, stop_psnr: float | None = None) -> dict:
    """Run the fit; PSNR every eval_every iterations. With stop_psnr, stop at
    the first evaluation that reaches it. Wall time counts the fit steps only."""
    curve = [(0, fit.psnr(eval_views))]
    wall = 0.0
    reached = None
    if stop_psnr is not None and curve[0][1] >= stop_psnr:
        reached = 0
    it = 0
    while it < iters and reached is None:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(eval_every):
            fit.step()
        torch.cuda.synchronize()
        wall += time.perf_counter() - t0
        it += eval_every
        p = fit.psnr(eval_views)
        curve.append((it, p))
        if stop_psnr is not None and p >= stop_psnr:
            reached = it
    return {"curve": curve, "iters": it, "wall_s": wall, "reached_at": reached, "final_psnr": curve[-1][1],
            "medium": fit.medium.cpu().numpy().tolist()}
