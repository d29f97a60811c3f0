"""Learned initial guess: data generation with the solver, training and
evaluation of the guess network (calls into libaxpcg only; PyTorch holds the
device arrays).

The network maps (log kappa, q, g / s) on an hw x hw lattice to u / s, where
g = B^-1 (r f) is the right-hand side after one application of the Laplace
preconditioner (the averaged-coefficient solution; `pre=False` uses f
itself) and s = max |g|; the network then only has to correct g for the
variable kappa.  The solver keeps the network's output as the starting
iterate only when that lowers the initial preconditioned residual
(AX_FLAG_CHECK_GUESS), and always iterates to the requested tolerance.
Training pairs come from solves of random-field media (workload 4); held-out
seeds come from a disjoint seed stream.
"""
from __future__ import annotations

import time

import numpy as np

from . import (AX_FLAG_CHECK_GUESS, AX_FLAG_USE_GUESS, AX_PCG_MIXED, AX_PREC_FP64, ax_apply_operator,
               ax_apply_preconditioner, ax_batch_create, ax_batch_destroy, ax_batch_solve, ax_destroy_operator,
               ax_guessnet_features, ax_guessnet_features_pre, ax_guessnet_forward, ax_guessnet_lift,
               ax_guessnet_train_step, ax_setup_operator, ax_solve)
from .inputs import sample_points


def grf_fields(specs, nr: int, nz: int, device):
    """kappa_r [n][nr][nz], kappa_z [n][nr][nz+1], q [n][nr][nz] and f [n][nr][nz]
    (FP64 torch tensors on `device`) of random-field media given by their
    specs (workloads.grf_spec), evaluated at the grid's sample points in bulk
    on the GPU."""
    import torch
    rn, rf, zn, zf = sample_points(nr, nz)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device)  # noqa: E731
    rn, rf, zn, zf = t(rn), t(rf), t(zn), t(zf)

    def field(spec, r, z):
        om, ph = t(spec["omega"]), t(spec["phase"])
        g = torch.zeros((r.numel(), z.numel()), dtype=torch.float64, device=device)
        for j0 in range(0, om.shape[0], 64):
            arg = (r[:, None, None] * om[None, None, j0:j0 + 64, 0] + z[None, :, None] * om[None, None, j0:j0 + 64, 1]
                   + ph[None, None, j0:j0 + 64])
            g += torch.cos(arg).sum(dim=2)
        g = spec["amp"] * g
        tt = ((g - spec["gmin"]) / (spec["gmax"] - spec["gmin"])).clamp(0.0, 1.0)
        return torch.exp(np.log(spec["contrast"]) * tt)

    kr, kz, qq, ff = [], [], [], []
    for sp in specs:
        kr.append(field(sp, rf, zn))
        kz.append(field(sp, rn, zf))
        qq.append(torch.full((nr, nz), sp["q"], dtype=torch.float64, device=device))
        f = torch.zeros((nr, nz), dtype=torch.float64, device=device)
        for rc, zc, sg, am in sp["sources"]:
            f += am * torch.exp(-((rn[:, None] - rc) ** 2 + (zn[None, :] - zc) ** 2) / (2 * sg * sg))
        ff.append(f)
    return torch.stack(kr), torch.stack(kz), torch.stack(qq), torch.stack(ff)


def large_fields(spec, nr: int, nz: int, device):
    """kappa_r [nr][nz], kappa_z [nr][nz+1], q [nr][nz] and f [M][nr][nz]
    (FP64 torch tensors on `device`) of a large layered medium given by its
    spec (workloads.large_spec), evaluated at the grid's sample points in
    bulk on the GPU: log kappa = log(layer value) + sum of the inclusions'
    log-factors times their logistic indicators, rescaled by the spec's
    extremes to [0, log contrast]; Gaussian sources."""
    import torch
    rn, rf, zn, zf = sample_points(nr, nz)
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64, device=device)  # noqa: E731
    rn, rf, zn, zf = t(rn), t(rf), t(zn), t(zf)
    cuts, values = t(spec["cuts"]), t(spec["values"])

    def kappa(r, z):
        lk = torch.log(values[torch.searchsorted(cuts, z, right=True)])[None, :].expand(r.numel(), z.numel())
        lk = lk.clone()
        for rc, zc, a, b, width, lf in spec["incs"]:
            rho = torch.sqrt(((r[:, None] - rc) / a) ** 2 + ((z[None, :] - zc) / b) ** 2)
            lk += lf * 0.5 * (1.0 - torch.tanh(0.5 * (rho - 1.0) * min(a, b) / width))
        tt = ((lk - spec["lmin"]) / (spec["lmax"] - spec["lmin"])).clamp(0.0, 1.0)
        return torch.exp(np.log(spec["contrast"]) * tt)

    sg = spec["sigma"]
    f = torch.stack([torch.exp(-((rn[:, None] - rc) ** 2 + (zn[None, :] - zc) ** 2) / (2 * sg * sg))
                     for rc, zc in spec["centres"]])
    q = torch.full((nr, nz), spec["q"], dtype=torch.float64, device=device)
    return kappa(rf, zn).contiguous(), kappa(rn, zf).contiguous(), q, f.contiguous()


def make_dataset_large(specs, nr: int, nz: int, hw: int, tol: float = 1e-8, device=None, target_scale: float = 0.0,
                       keep_ops: bool = False):
    """Solves every large medium (all its right-hand sides at once, mixed
    PCG) and returns the lattice features x [n][3][hw][hw], the targets u / s
    averaged over hw x hw cells (FP32, scaled by tscale), the scales s and
    the solves' iteration counts; with keep_ops, the operators and the fields
    stay for evaluation (one medium at a time otherwise, to bound memory)."""
    import torch
    xs, ys, ss, iters, kept = [], [], [], [], []
    for spec in specs:
        kr, kz, q, f = large_fields(spec, nr, nz, device)
        m = f.shape[0]
        op = ax_setup_operator(kr, kz, q, nr, nz)
        u = torch.zeros_like(f)
        _, info = ax_solve(op, f, u, m, tol, 20000, AX_PCG_MIXED)
        iters += [i["iters"] for i in info]
        x = torch.zeros((m, 3, hw, hw), dtype=torch.float32, device=device)
        s = torch.zeros(m, dtype=torch.float64, device=device)
        ax_guessnet_features_pre(op, kr, q, f, m, hw, x, s)
        y = torch.nn.functional.avg_pool2d((u / s[:, None, None]).float()[:, None], (nr // hw, nz // hw))[:, 0]
        xs.append(x)
        ys.append(y)
        ss.append(s)
        if keep_ops:
            kept.append({"op": op, "kr": kr, "q": q, "f": f, "u": u, "iters": [i["iters"] for i in info]})
        else:
            ax_destroy_operator(op)
            del kr, kz, q, f, u
    x, y, s = torch.cat(xs), torch.cat(ys), torch.cat(ss)
    tscale = target_scale if target_scale else float(1.0 / y.std().item())
    return {"x": x, "y": (y * tscale).contiguous(), "s": s, "iters": iters, "tscale": tscale, "media": kept}


def guess_large(net: int, medium, hw: int, nr: int, nz: int, tscale: float):
    """u0 [M][nr][nz] for every right-hand side of a kept large medium:
    features (with the preconditioned right-hand side) -> network (one batch)
    -> bilinear lift -> scale."""
    import torch
    dev = medium["f"].device
    m = medium["f"].shape[0]
    x = torch.zeros((m, 3, hw, hw), dtype=torch.float32, device=dev)
    s = torch.zeros(m, dtype=torch.float64, device=dev)
    ax_guessnet_features_pre(medium["op"], medium["kr"], medium["q"], medium["f"], m, hw, x, s)
    y = torch.zeros((m, hw, hw), dtype=torch.float32, device=dev)
    ax_guessnet_forward(net, x, y, m)
    u0 = torch.zeros_like(medium["f"])
    ax_guessnet_lift(y, m, hw, s / tscale, nr, nz, u0)
    return u0


def _features(data, i, x, s):
    """Features of sample i into x [1][3][hw][hw] and its scale into s [1]."""
    hw = x.shape[-1]
    if data["pre"]:
        ax_guessnet_features_pre(data["ops"][i], data["kr"][i], data["q"][i], data["f"][i], 1, hw, x, s)
    else:
        nr, nz = data["f"].shape[1:]
        ax_guessnet_features(data["kr"][i], data["q"][i], data["f"][i], 1, nr, nz, hw, x, s)


def make_dataset(specs, nr: int, nz: int, hw: int, tol: float = 1e-8, device=None, target_scale: float = 0.0,
                 pre: bool = True):
    """Solves every medium with the batched solver and returns features x
    [n][3][hw][hw], targets u / s [n][hw][hw] (FP32 torch tensors), the
    operators' inputs and the solutions (FP64)."""
    import torch
    kr, kz, q, f = grf_fields(specs, nr, nz, device)
    n = len(specs)
    ops = [ax_setup_operator(kr[i], kz[i], q[i], nr, nz) for i in range(n)]
    u = torch.zeros_like(f)
    batch = ax_batch_create(ops)
    _, info = ax_batch_solve(batch, [f[i] for i in range(n)], [u[i] for i in range(n)], tol, 20000, AX_PCG_MIXED)
    ax_batch_destroy(batch)
    x = torch.zeros((n, 3, hw, hw), dtype=torch.float32, device=device)
    s = torch.zeros(n, dtype=torch.float64, device=device)
    data = {"kr": kr, "q": q, "f": f, "ops": ops, "pre": pre}
    for i in range(n):
        _features(data, i, x[i:i + 1], s[i:i + 1])
    # targets on the lattice: cell averages of u / s (the lattice equals the grid
    # here when nr = nz = hw)
    if nr == hw and nz == hw:
        y = (u / s[:, None, None]).float()
    else:
        y = torch.nn.functional.avg_pool2d((u / s[:, None, None]).float()[:, None], (nr // hw, nz // hw))[:, 0]
    # u / s is small (~1e-3); the network learns the target scaled to unit
    # spread, and its output is divided by the same factor at solve time
    tscale = target_scale if target_scale else float(1.0 / y.std().item())
    data.update({"x": x, "y": (y * tscale).contiguous(), "kz": kz, "u": u, "s": s,
                 "iters": [i["iters"] for i in info], "tscale": tscale})
    return data


def train(net: int, data, epochs: int, batch: int, lr: float, seed: int = 0, log=None):
    import torch
    n = data["x"].shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(n)
        ep_loss = 0.0
        steps = 0
        for k in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(order[k:k + batch], device=data["x"].device)
            xb = data["x"].index_select(0, idx).contiguous()
            yb = data["y"].index_select(0, idx).contiguous()
            ep_loss += ax_guessnet_train_step(net, xb, yb, batch, lr * (0.5 ** (ep // max(1, epochs // 3))))
            steps += 1
        losses.append(ep_loss / max(1, steps))
        if log:
            log(f"epoch {ep} loss {losses[-1]:.4e}")
    return losses


def guess_for(net: int, data, i: int, hw: int, nr: int, nz: int):
    """u0 for sample i: features -> network -> bilinear lift -> scale."""
    import torch
    dev = data["f"].device
    x = torch.zeros((1, 3, hw, hw), dtype=torch.float32, device=dev)
    s = torch.zeros(1, dtype=torch.float64, device=dev)
    _features(data, i, x, s)
    y = torch.zeros((1, hw, hw), dtype=torch.float32, device=dev)
    ax_guessnet_forward(net, x, y, 1)
    u0 = torch.zeros((1, nr, nz), dtype=torch.float64, device=dev)
    ax_guessnet_lift(y, 1, hw, s / data["tscale"], nr, nz, u0)
    return u0


def energy_ratio(op, f, u0):
    """sqrt((r0, B^-1 r0) / (phi, B^-1 phi)) for r0 = phi - A u0, phi = r f: the
    quantity the solver's guess gate compares with 1 (diagnostic, FP64)."""
    import torch
    from .inputs import sample_points
    nr, nz = f.shape[-2:]
    rn = torch.as_tensor(sample_points(nr, nz)[0], dtype=torch.float64, device=f.device)
    phi = (rn[:, None] * f.reshape(nr, nz)).reshape(1, nr, nz).contiguous()
    au = torch.zeros_like(phi)
    ax_apply_operator(op, u0.reshape(1, nr, nz).contiguous(), au, 1, AX_PREC_FP64)
    r0 = phi - au
    br, bp = torch.zeros_like(phi), torch.zeros_like(phi)
    ax_apply_preconditioner(op, r0, br, 1, AX_PREC_FP64)
    ax_apply_preconditioner(op, phi, bp, 1, AX_PREC_FP64)
    return float(torch.sqrt((r0 * br).sum() / (phi * bp).sum()))


def energy_error_ratio(op, u, u0):
    """||u0 - u||_A / ||u||_A (A in FP64) for the converged solution u: the
    initial error in the norm that bounds PCG's convergence (diagnostic)."""
    import torch
    nr, nz = u.shape[-2:]
    e = (u0 - u).reshape(1, nr, nz).contiguous()
    uu = u.reshape(1, nr, nz).contiguous()
    ae, au = torch.zeros_like(e), torch.zeros_like(e)
    ax_apply_operator(op, e, ae, 1, AX_PREC_FP64)
    ax_apply_operator(op, uu, au, 1, AX_PREC_FP64)
    return float(torch.sqrt((e * ae).sum() / (uu * au).sum()))


def lattice_bounds(op, f, u, hw: int):
    """What any guess built on an hw x hw lattice can reach, per right-hand
    side of f [M][nr][nz] with converged solutions u (diagnostic, FP64
    operator): the energy-norm error ratio ||u0 - u||_A / ||u||_A of
    (a) the bilinear lift of u's own cell averages, (b) one preconditioned
    step from zero, u0 = a g with g = B^-1 (r f) and the A-optimal a, and
    (c) that step plus the lift of the cell averages of its remainder u - a g."""
    import torch
    from .inputs import sample_points
    m, nr, nz = f.shape
    rn = torch.as_tensor(sample_points(nr, nz)[0], dtype=torch.float64, device=f.device)
    out = {"lattice": [], "one_step": [], "one_step_plus_lattice": []}
    ones = torch.ones(1, dtype=torch.float64, device=f.device)

    def lift_avg(v):
        y = torch.nn.functional.avg_pool2d(v.float()[None, None], (nr // hw, nz // hw))[0].contiguous()
        w = torch.zeros((1, nr, nz), dtype=torch.float64, device=f.device)
        ax_guessnet_lift(y, 1, hw, ones, nr, nz, w)
        return w[0]

    for j in range(m):
        phi = (rn[:, None] * f[j]).reshape(1, nr, nz).contiguous()
        g = torch.zeros_like(phi)
        ax_apply_preconditioner(op, phi, g, 1, AX_PREC_FP64)
        ag = torch.zeros_like(phi)
        ax_apply_operator(op, g, ag, 1, AX_PREC_FP64)
        a = float((g * phi).sum() / (g * ag).sum())
        ug = a * g[0]
        out["lattice"].append(energy_error_ratio(op, u[j], lift_avg(u[j])))
        out["one_step"].append(energy_error_ratio(op, u[j], ug))
        out["one_step_plus_lattice"].append(energy_error_ratio(op, u[j], ug + lift_avg(u[j] - ug)))
    return out


def evaluate(net: int, data, hw: int, nr: int, nz: int, tol: float = 1e-8, method: int = AX_PCG_MIXED):
    """Per held-out sample: iterations and wall time from zero and from the
    network's guess (guess time included), with the residual gate on, and
    the guess's gate ratio (energy_ratio)."""
    import torch
    rows = []
    for i, op in enumerate(data["ops"]):
        f = data["f"][i:i + 1]
        u = torch.zeros_like(f)
        ax_solve(op, f, u, 1, tol, 20000, method)          # warm the graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u.zero_()
        _, i0 = ax_solve(op, f, u, 1, tol, 20000, method)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u0 = guess_for(net, data, i, hw, nr, nz)
        _, ig = ax_solve(op, f, u0, 1, tol, 20000, method, AX_FLAG_USE_GUESS | AX_FLAG_CHECK_GUESS)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        rows.append({"iters_zero": i0[0]["iters"], "iters_guess": ig[0]["iters"], "ms_zero": 1e3 * (t1 - t0),
                     "ms_guess": 1e3 * (t2 - t1), "accepted": ig[0]["guess_accepted"],
                     "res_zero": i0[0]["rel_res"], "res_guess": ig[0]["rel_res"],
                     "energy_ratio": energy_ratio(op, f, guess_for(net, data, i, hw, nr, nz))})
    return rows


def release(data):
    for op in data["ops"]:
        ax_destroy_operator(op)
    data["ops"] = []
