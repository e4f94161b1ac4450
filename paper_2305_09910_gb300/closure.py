"""Learned closure workflow: data from fine runs, training, and the a-posteriori comparison.

Every arithmetic step runs in the library's kernels (lbm_closure_samples, lbm_filter2,
lbm_closure_loss_grad, lbm_adam_step, the fused closure in the collide kernel, the FP64
statistics); this module only sequences them and holds tensors.  Host-side numpy is used
for the evaluation summaries (profile errors) and to choose the feature scales.

Grids (acoustic scaling, box filter of width 2): the fine channel has twice the cells of the
coarse one in every axis; one coarse step spans two fine steps; velocities are equal in
lattice units; nu_c = nu_f / 2 and the body force per unit mass g_c = 2 g_f.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, lbm

FACES_CHANNEL = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")
NP = lbm.MLP_NPARAM
# offsets of the output layer (W3, b3) in the packed parameter vector
OUT_LAYER = slice(32 * 7 + 32 + 32 * 32 + 32, NP)


def channel(nx, ny, nz, closure="smag", cs0=0.1, precision="f32", re_tau=180.0, u_bulk=0.05,
            seed=inputs.DEFAULT_SEED, tau=None, force=None, amp=0.1, streaming="aa"):
    """A channel lattice (walls at the y faces) initialised from the perturbed parabola."""
    import torch

    par = inputs.channel_parameters(ny, re_tau=re_tau, u_bulk=u_bulk)
    tau = par["tau"] if tau is None else tau
    force = par["force"] if force is None else force
    lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=tau, precision=precision, closure=closure,
                      cs_smag=cs0, faces=FACES_CHANNEL, streaming=streaming)
    lat.set_force(force)
    rho = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    step = max(1, nz // 8)
    for z0 in range(0, nz, step):  # slab by slab to bound host memory
        z1 = min(nz, z0 + step)
        r, v = inputs.channel_init(nx, ny, nz, u_bulk=u_bulk, seed=seed, z_range=(z0, z1), amp=amp)
        rho[z0:z1].copy_(torch.from_numpy(r))
        u[:, z0:z1].copy_(torch.from_numpy(v))
    lat.init_equilibrium(rho, u)
    lat.tau, lat.force = tau, force
    return lat


class Samples:
    """Training pairs on the GPU: x (n, 7), target nu*, |S_c|, weight |S_c|^2."""

    def __init__(self, n):
        import torch

        self.x = torch.zeros((n, 7), dtype=torch.float32, device="cuda")
        self.target = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.smag = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.weight = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.n = 0

    def tensors(self):
        return self.x, self.target, self.smag, self.weight


def feature_scales(fine, tau0_c, cs0):
    """1 / standard deviation of the stress features and of rho - 1 on one snapshot."""
    nc = fine.ncell // 8
    s = Samples(nc)
    lbm.lbm_closure_samples(fine.h, tau0_c, cs0, (1.0, 1.0), *s.tensors())
    x = s.x.cpu().numpy().astype(np.float64)
    sd_pi = float(np.sqrt((x[:, :6] ** 2).mean()))
    sd_rho = float(x[:, 6].std())
    return (1.0 / max(sd_pi, 1e-30), 1.0 / max(sd_rho, 1e-12))


def collect(fine, tau0_c, cs0, scale, nsnap, every, samples=None):
    """Runs the fine lattice and appends one set of coarse samples every `every` steps."""
    nc = fine.ncell // 8
    if samples is None:
        samples = Samples(nc * nsnap)
    for _ in range(nsnap):
        fine.step(every)
        a, b = samples.n, samples.n + nc
        lbm.lbm_closure_samples(fine.h, tau0_c, cs0, scale, samples.x[a:b], samples.target[a:b],
                                samples.smag[a:b], samples.weight[a:b])
        samples.n = b
    fine.sync()
    return samples


def init_params(seed=0):
    """Random hidden layers, zero output layer: starts exactly at Smagorinsky (y = 0)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NP, dtype=np.float32)
    p[: 32 * 7] = rng.normal(0, 1 / math.sqrt(7), 32 * 7)
    p[32 * 7 + 32: 32 * 7 + 32 + 1024] = rng.normal(0, 1 / math.sqrt(32), 1024)
    return p


def loss(params, samples, cs0, first=0, n=None, stride=1):
    import torch

    n = (samples.n - first) // stride if n is None else n
    g = torch.zeros(NP, dtype=torch.float32, device="cuda")
    return lbm.lbm_closure_loss_grad(params, *samples.tensors(), n, first, stride, cs0, g)


def train(samples, cs0, epochs=4, nbatch=64, lr=2e-3, seed=0, params=None, log=None):
    """Adam on interleaved minibatches (batch b = samples b, b + nbatch, ...)."""
    import torch

    p = torch.from_numpy(init_params(seed) if params is None else params).cuda()
    g = torch.zeros(NP, dtype=torch.float32, device="cuda")
    m = torch.zeros(NP, dtype=torch.float32, device="cuda")
    v = torch.zeros(NP, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    n_b = samples.n // nbatch
    t = 0
    history = []
    for ep in range(epochs):
        tot = 0.0
        for b in rng.permutation(nbatch):
            t += 1
            tot += lbm.lbm_closure_loss_grad(p, *samples.tensors(), n_b, int(b), nbatch, cs0, g)
            lbm.lbm_adam_step(p, g, m, v, lr * (0.5 ** (ep // 2)), t)
        history.append(tot / nbatch)
        if log:
            log(f"epoch {ep}: mean minibatch loss {history[-1]:.4e}")
    return p, history


def profiles(stats, nsamples):
    """Mean u_x and RMS (u_x', u_y', u_z') per y plane from LBM_STATS_K sums."""
    cnt = np.maximum(stats[:, 0], 1.0)
    mean = stats[:, 1:4] / cnt[:, None]
    sq = stats[:, 4:7] / cnt[:, None]
    rms = np.sqrt(np.maximum(sq - mean ** 2, 0.0))
    return mean[:, 0], rms


def filtered_profiles(fine, rb, ub):
    """The same profiles of the box-filtered fine velocity (accumulated by the caller)."""
    lbm.lbm_filter2(fine.h, rb, ub)
    u = ub.cpu().numpy().astype(np.float64)  # (3, nzc, nyc, nxc)
    return u.mean(axis=(1, 3)), (u * u).mean(axis=(1, 3))


def aposteriori(fine, params, scale, cs0, coarse_steps, every=10, log=None, cs_min=0.0):
    """Coarse runs (Smagorinsky and learned closure) from the filtered fine state, against the
    filtered fine run over the same physical time.  Returns relative profile errors."""
    import torch

    nxc, nyc, nzc = fine.nx // 2, fine.ny // 2, fine.nz // 2
    nc = nxc * nyc * nzc
    rb = torch.zeros((nzc, nyc, nxc), dtype=torch.float32, device="cuda")
    ub = torch.zeros((3, nzc, nyc, nxc), dtype=torch.float32, device="cuda")
    lbm.lbm_filter2(fine.h, rb, ub)
    nu_f = (fine.tau - 0.5) / 3.0
    tau_c = 3.0 * nu_f / 2.0 + 0.5
    runs = {}
    for name in ("smag", "mlp"):
        lat = lbm.Lattice(nxc, nyc, nzc, stencil=19, tau=tau_c, closure=name, cs_smag=cs0,
                          faces=FACES_CHANNEL)
        lat.set_force(2.0 * fine.force)
        if name == "mlp":
            lbm.lbm_set_closure_f32(lat.h, params, *scale)
            lbm.lbm_set_closure_floor(lat.h, cs_min)
        lat.init_equilibrium(rb, ub)
        lbm.lbm_stats_reset(lat.h)
        runs[name] = lat
    ref_m = np.zeros((nyc, 3))
    ref_q = np.zeros((nyc, 3))
    nref = 0
    t0 = time.time()
    for k in range(coarse_steps // every):
        for lat in runs.values():
            lat.step(every)
            lbm.lbm_stats_sample(lat.h)
        fine.step(2 * every)
        m, q = filtered_profiles(fine, rb, ub)
        ref_m += m.T
        ref_q += q.T
        nref += 1
    out = {"coarse_steps": coarse_steps, "wall_s": time.time() - t0}
    ref_mean = ref_m / nref
    ref_rms = np.sqrt(np.maximum(ref_q / nref - ref_mean ** 2, 0.0))
    for name, lat in runs.items():
        try:
            lat.sync()
        except lbm.LbmError as e:
            if e.status != lbm.LBM_EUNSTABLE:
                raise
            out[name] = {"unstable": True}
            lat.close()
            continue
        st, ns = lbm.lbm_stats_get(lat.h, nyc)
        mean, rms = profiles(st, ns)
        e_mean = float(np.linalg.norm(mean - ref_mean[:, 0]) / np.linalg.norm(ref_mean[:, 0]))
        e_rms = float(np.linalg.norm(rms - ref_rms) / max(np.linalg.norm(ref_rms), 1e-30))
        out[name] = {"mean_err": e_mean, "rms_err": e_rms, "samples": ns}
        lat.close()
    out["ref_rms_max"] = float(ref_rms.max())
    if log:
        log(f"a posteriori: {out}")
    return out


def split(samples, frac):
    """(train, held-out) views: the first `frac` of the samples (earlier snapshots) and the rest."""
    n = int(samples.n * frac)
    a, b = Samples.__new__(Samples), Samples.__new__(Samples)
    a.x, a.target, a.smag, a.weight, a.n = (samples.x[:n], samples.target[:n], samples.smag[:n],
                                            samples.weight[:n], n)
    b.x, b.target, b.smag, b.weight, b.n = (samples.x[n:], samples.target[n:], samples.smag[n:],
                                            samples.weight[n:], samples.n - n)
    return a, b


def experiment(nx, ny, nz, re_tau=180.0, u_bulk=0.05, spin=60000, nsnap=20, every=500, epochs=6,
               coarse_steps=20000, cs0=0.1, cs_min=0.1, seed=0, log=None, amp=0.1, flow_seed=None):
    """The learned-closure experiment on a fine channel of nx x ny x nz cells.

    1. spin the fine Smagorinsky channel up; 2. collect nsnap box-filtered sample sets;
    3. train on the first 3/4 (earlier snapshots), score on the last 1/4 against Smagorinsky
    (the zero output layer); 4. from the filtered final fine state, run the coarse channel
    with Smagorinsky and with the learned closure (bounded below by cs_min) and compare
    their mean and RMS velocity profiles with the filtered fine run over the same time.
    `seed` seeds the network's initial weights and the minibatch order, `flow_seed` (default
    the inputs' default seed) the perturbations of the initial channel state."""
    import torch

    t0 = time.time()
    rep = {"fine": [nx, ny, nz], "coarse": [nx // 2, ny // 2, nz // 2], "re_tau": re_tau,
           "u_bulk": u_bulk, "spin_steps": spin, "snapshots": nsnap, "every": every,
           "epochs": epochs, "coarse_steps": coarse_steps, "cs0": cs0, "cs_min": cs_min}
    flow_seed = inputs.DEFAULT_SEED if flow_seed is None else flow_seed
    rep["flow_seed"] = flow_seed
    fine = channel(nx, ny, nz, closure="smag", cs0=cs0, re_tau=re_tau, u_bulk=u_bulk, amp=amp, seed=flow_seed)
    fine.step(spin)
    fine.sync()
    lbm.lbm_stats_reset(fine.h)
    lbm.lbm_stats_sample(fine.h)
    st, _ = lbm.lbm_stats_get(fine.h, ny)
    rep["fine_rms_max_after_spin"] = profiles(st, 1)[1].max(axis=0).tolist()
    rep["amp"] = amp
    tau_c = 1.5 * (fine.tau - 0.5) / 3.0 + 0.5
    rep["tau_fine"], rep["tau_coarse"] = fine.tau, tau_c
    scale = feature_scales(fine, tau_c, cs0)
    rep["scale"] = list(scale)
    samples = collect(fine, tau_c, cs0, scale, nsnap, every)
    tr, ho = split(samples, 0.75)
    p, hist = train(tr, cs0, epochs=epochs, seed=seed, log=log)
    base = torch.from_numpy(init_params(seed)).cuda()  # zero output layer = Smagorinsky
    rep["train_loss"] = hist
    rep["heldout_loss_smag"] = loss(base, ho, cs0)
    rep["heldout_loss_mlp"] = loss(p, ho, cs0)
    rep["apriori_gain"] = 1.0 - rep["heldout_loss_mlp"] / rep["heldout_loss_smag"]
    rep["t_train_s"] = time.time() - t0
    rep["aposteriori"] = aposteriori(fine, p, scale, cs0, coarse_steps, every=10, log=log, cs_min=cs_min)
    rep["params"] = p.cpu().numpy().tolist()
    rep["wall_s"] = time.time() - t0
    if log:
        log(f"experiment done in {rep['wall_s']:.1f} s: a-priori gain {rep['apriori_gain']:.3f}")
    return rep


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="learned-closure experiment (fine run, training, coarse comparison)")
    ap.add_argument("--size", default="512x256x256", help="fine lattice NXxNYxNZ")
    ap.add_argument("--re-tau", type=float, default=180.0)
    ap.add_argument("--u-bulk", type=float, default=0.05)
    ap.add_argument("--spin", type=int, default=150000)
    ap.add_argument("--snapshots", type=int, default=200)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--coarse-steps", type=int, default=20000)
    ap.add_argument("--cs-min", type=float, default=0.1)
    ap.add_argument("--amp", type=float, default=0.1, help="sinusoid amplitude / u_bulk")
    ap.add_argument("--out", default=None, help="JSON report path")
    a = ap.parse_args()
    nx, ny, nz = (int(v) for v in a.size.split("x"))
    rep = experiment(nx, ny, nz, a.re_tau, a.u_bulk, a.spin, a.snapshots, a.every, a.epochs,
                     a.coarse_steps, cs_min=a.cs_min, log=lambda s: print(s, flush=True), amp=a.amp)
    short = {k: v for k, v in rep.items() if k != "params"}
    print(json.dumps(short))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(rep, fh)
