"""The learned troubled-cell indicator, end to end: labels from the TVB test on
the method's own runs, training on the GPU with libdg's kernels, and the
measures that compare it with the TVB test it stands in for.

Labels.  A TVB-limited run (limiter 1, positivity) of the disc is sampled
every few steps; each sampled state takes one step without troubled-cell
limiting (positivity kept) on a scratch handle, and the TVB test of that
unlimited value gives the labels -- the kind of value the limiter flags after
every stage.  Every troubled element is kept, with a seeded sample of as many
(times `neg_ratio`) untroubled ones.

Measures.  On held-out states: miss rate P(net 0 | TVB 1) and false-flag
rate P(net 1 | TVB 0).  Induced solution error: runs from the same initial
data with the TVB test (limiter 1), the network (limiter 2) and no
troubled-cell limiting (positivity only); relative L2 of the density of the
last two against the first.
"""
import copy
import time

import numpy as np

from . import dg


def _cfg(cfg, limiter, positivity=1):
    c = copy.deepcopy(cfg)
    c["disc"]["limiter"] = limiter
    c["disc"]["positivity"] = positivity
    return c


def labelled_states(cfg, snapshots, every, M, neg_ratio=1.0, seed=0):
    """Features (torch CUDA [n, nin]) and labels (torch CUDA [n]) from a
    TVB-limited run of `cfg`."""
    import torch
    rng = np.random.default_rng(seed)
    run = dg.Disc(_cfg(cfg, 1))
    scratch = dg.Disc(_cfg(cfg, 0))
    X, Y, stats = [], [], []
    try:
        for _ in range(snapshots):
            run.step(every)
            t, _, st = run.get_time()
            scratch.set_state(run.fetch(), t, st)
            scratch.step(1)
            flags = scratch.indicator(M).ravel()
            pos = np.flatnonzero(flags)
            neg_all = np.flatnonzero(flags == 0)
            nneg = min(neg_all.size, max(int(neg_ratio * pos.size), 64))
            neg = rng.choice(neg_all, size=nneg, replace=False)
            elems = np.concatenate([pos, neg]).astype(np.int32)
            X.append(scratch.features(torch.from_numpy(elems).cuda()))
            Y.append(torch.from_numpy(flags[elems].astype(np.float32)).cuda())
            stats.append((int(pos.size), int(flags.size)))
    finally:
        run.close()
        scratch.close()
    return torch.cat(X), torch.cat(Y), stats


def train(X, Y, epochs=20, batch=4096, lr=2e-3, seed=0):
    """A dg.Mlp trained on (X, Y) with Adam, the positive class weighted by
    the class ratio; returns (net, losses per epoch, seconds)."""
    import torch
    net = dg.Mlp(X.shape[1], seed=seed)
    n = X.shape[0]
    npos = float(Y.sum().item())
    pw = max((n - npos) / max(npos, 1.0), 1.0)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot, cnt = 0.0, 0
        for k in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = perm[k:k + batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            tot += net.train_step(xb, yb, pos_weight=pw, lr=lr) * xb.shape[0]
            cnt += xb.shape[0]
        losses.append(tot / max(cnt, 1))
    torch.cuda.synchronize()
    return net, losses, time.perf_counter() - t0


def calibrate(net, X, Y, miss=0.005):
    """The largest threshold whose miss rate on the training examples is at
    most `miss` (the false flags fall as the threshold rises)."""
    import torch
    z = net.forward(X)
    zp = z[Y > 0.5]
    if zp.numel() == 0:
        return 0.0
    return float(torch.quantile(zp.float().cpu(), miss).item())


def rates(net, cfg, snapshots, every, M, threshold=0.0):
    """Miss and false-flag rates of `net` against the TVB test on the
    labelled states of a run of `cfg` (all elements)."""
    run = dg.Disc(_cfg(cfg, 1))
    scratch = dg.Disc(_cfg(cfg, 0))
    miss = hit = false = neg = 0
    try:
        scratch.set_indicator(net, threshold)
        for _ in range(snapshots):
            run.step(every)
            t, _, st = run.get_time()
            scratch.set_state(run.fetch(), t, st)
            scratch.step(1)
            tvb = scratch.indicator(M).astype(bool)
            _, f = scratch.indicator_logits()
            f = f.astype(bool)
            miss += int((tvb & ~f).sum())
            hit += int(tvb.sum())
            false += int((f & ~tvb).sum())
            neg += int((~tvb).sum())
    finally:
        run.close()
        scratch.close()
    return {"miss_rate": miss / max(hit, 1), "false_flag_rate": false / max(neg, 1),
            "troubled": hit, "untroubled": neg}


def inference_ms(net, cfg, reps=5, threshold=0.0):
    """Mean time of one fused inference pass over every element of a state of
    `cfg` (features on the fly, flags), CUDA events."""
    import torch
    d = dg.Disc(_cfg(cfg, 2))
    try:
        d.set_indicator(net, threshold)
        d.indicator_logits()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            d.limit()  # limiter 2: network flags, then the limited reduction
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps
    finally:
        d.close()


def evaluate(cfg_train, cfg_rates, cfg_err, *, snapshots=12, every=6, M=50.0, epochs=60, err_steps=40,
             neg_ratio=8.0, seed=1):
    """Labels, training, calibration and the measures, as one record."""
    t0 = time.perf_counter()
    X, Y, stats = labelled_states(cfg_train, snapshots, every, M, neg_ratio=neg_ratio, seed=seed)
    t1 = time.perf_counter()
    net, losses, t_train = train(X, Y, epochs=epochs, seed=seed)
    thr = calibrate(net, X, Y)
    r = rates(net, cfg_rates, 4, every, M, thr)
    err = induced_error(net, cfg_err, err_steps, thr)
    ms_inf = inference_ms(net, cfg_err, threshold=thr)
    out = {"examples": int(X.shape[0]), "troubled_examples": int(Y.sum().item()),
           "label_seconds": t1 - t0, "train_seconds": t_train, "epochs": epochs,
           "final_loss": losses[-1], "threshold": thr, **r, "runs": err,
           "limit_pass_ms_with_network": ms_inf}
    net.close()
    return out


def induced_error(net, cfg, steps, threshold=0.0):
    """Density of the network-limited and of the unlimited (positivity only)
    runs against the TVB-limited run after `steps` steps, relative L2, and
    the mean step time of each run."""
    import torch
    out = {}
    ref = None
    for name, lim in (("tvb", 1), ("mlp", 2), ("none", 0)):
        d = dg.Disc(_cfg(cfg, lim))
        try:
            if lim == 2:
                d.set_indicator(net, threshold)
            d.step(1)
            d.sync()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d.step(steps - 1)
            d.sync()
            ms = (time.perf_counter() - t0) * 1e3 / max(steps - 1, 1)
            sig = d.fetch()[0]
        finally:
            d.close()
        if ref is None:
            ref = sig
        out[name] = {"ms_per_step": ms,
                     "rel_l2_sigma_vs_tvb": float(np.linalg.norm(sig - ref) / np.linalg.norm(ref))}
    return out


def limit_pass_ms(n=1024, order=3, reps=5, warmup=2):
    """Mean time in ms of one limit pass with a seeded untrained network
    (limiter 2; the kernels' work does not depend on the weights) on the n^2
    shock-ring disc of degree `order`, timed with CUDA events over `reps`
    passes after `warmup` untimed ones."""
    import torch
    from . import inputs
    cfg = inputs.shock_ring(n, order)
    cfg["disc"]["limiter"] = 2
    d = dg.Disc(cfg)
    net = dg.Mlp(5 * 4 * (order + 1) ** 2, seed=1)
    try:
        d.set_indicator(net, 0.0)
        for _ in range(warmup):
            d.limit()
        d.sync()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            d.limit()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / max(reps, 1)
    finally:
        net.close()
        d.close()
