"""Training and use of the convolutional surrogate of 64 LBM steps.

The network itself (mlswlbm_surrogate_*, BF16 tensor-core kernels) lives in
the C library; this module feeds it:

* trajectories: the heights of many instances of one lattice after every
  window of 64 steps, run by one batch of the solver;
* training: Adam on random minibatches of (h(t), h(t + 64)) pairs;
* evaluation: the largest height error of each window against the LBM, next
  to that of the identity map (no change);
* rollout: an instance advanced window by window, by the surrogate where an
  acceptance rule calibrated on training windows says its height error
  stays within a bound, by the LBM elsewhere.

Device arrays are float32 torch CUDA tensors [.., n, ny, nx].
"""
import time

import numpy as np

from . import mlswlbm as B

WINDOW = 64  # LBM steps per surrogate call


def _torch():
    import torch
    return torch


def trajectories(params, heights, windows, stream=None):
    """Heights after 0..windows windows of every instance (all of one shape):
    a tensor [instances][windows + 1][n][ny][nx] on the GPU."""
    torch = _torch()
    p0 = params[0]
    n, ny, nx = int(p0["n"]), int(p0["ny"]), int(p0["nx"])
    out = torch.empty((len(params), windows + 1, n, ny, nx), dtype=torch.float32, device="cuda")
    host = np.empty((n, ny, nx), dtype=np.float32)
    with B.Batch(params, heights, stream=stream) as b:
        for w in range(windows + 1):
            if w:
                b.step(WINDOW)
            for j in range(len(params)):
                b.get_heights(j, host)
                out[j, w].copy_(torch.from_numpy(host))
        if b.status() != B.MLSW_OK:
            raise RuntimeError("solver status: " + B.mlswlbm_strerror(b.status()))
    return out


def train(s, traj, instances, steps, batch, lr, lr_end=None, seed=0, weights=None):
    """Adam steps on minibatches of windows of the given instances; the
    learning rate decays geometrically from lr to lr_end. `weights`
    (optional, one per window index) sets how often each window is drawn.
    Returns the losses."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    nwin = traj.shape[1] - 1
    inst = np.asarray(instances)
    lr_end = lr if lr_end is None else lr_end
    prob = None if weights is None else np.asarray(weights, dtype=float) / np.sum(weights)
    losses = []
    for it in range(steps):
        ii = torch.as_tensor(rng.choice(inst, batch), device="cuda")
        ww = torch.as_tensor(rng.choice(nwin, batch, p=prob), device="cuda")
        h = traj[ii, ww].contiguous()
        t = traj[ii, ww + 1].contiguous()
        rate = lr * (lr_end / lr) ** (it / max(steps - 1, 1))
        losses.append(s.train_step(h, t, rate))
    return np.array(losses)


def window_errors(s, traj, instances):
    """Per (instance, window): the surrogate's largest height error against
    the LBM, that of the identity map, and the surrogate's predicted largest
    change. Arrays [instances][windows]."""
    torch = _torch()
    errs, ident, change = [], [], []
    for i in instances:
        h_all, t_all = traj[i, :-1], traj[i, 1:]
        e, c = [], []
        for k in range(0, h_all.shape[0], s.max_batch):
            h = h_all[k:k + s.max_batch].contiguous()
            pred = torch.empty_like(h)
            s.predict(h, pred)
            e.append((pred - t_all[k:k + s.max_batch]).abs().amax(dim=(1, 2, 3)))
            c.append((pred - h).abs().amax(dim=(1, 2, 3)))
        errs.append(torch.cat(e).cpu().numpy())
        change.append(torch.cat(c).cpu().numpy())
        ident.append((t_all - h_all).abs().amax(dim=(1, 2, 3)).cpu().numpy())
    return np.array(errs), np.array(ident), np.array(change)


def calibrate(err, change, bound=1e-3, quantile=1.0):
    """Largest threshold tau on the predicted change such that, among the
    windows whose predicted change is at most tau, a fraction `quantile` has
    an error within `bound` (0 if none qualifies)."""
    order = np.argsort(change.ravel())
    e = err.ravel()[order]
    c = change.ravel()[order]
    ok = np.cumsum(e <= bound) / np.arange(1, e.size + 1)
    good = np.nonzero(ok >= quantile)[0]
    return float(c[good[-1]]) if good.size else 0.0


def rollout(s, params, h0, windows, tau, hand_over=False):
    """Advances one instance by `windows` windows: the surrogate's window is
    taken when its predicted largest change is at most tau, otherwise the LBM
    runs the 64 steps, restarted from the current heights (all on the
    device; one host read of the predicted change per window). A restart
    sets the populations to f_eq(h, U = 0): the layer fluxes of the previous
    LBM window are not carried over, so the LBM windows of a rollout are
    not the uninterrupted LBM trajectory from the same heights. With
    hand_over, the first window the surrogate does not take hands all the
    remaining windows to the LBM in one call (a film whose change has grown
    past tau keeps changing faster until it has dewetted). Returns (heights,
    windows taken from the surrogate, seconds)."""
    torch = _torch()
    n, ny, nx = int(params["n"]), int(params["ny"]), int(params["nx"])
    h = torch.from_numpy(np.asarray(h0, dtype=np.float32).reshape(1, n, ny, nx)).cuda()
    pred = torch.empty_like(h)
    taken = 0
    with B.Solver(params, np.asarray(h0, dtype=np.float32),
                  stream=torch.cuda.current_stream()) as lbm:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for w in range(windows):
            s.predict(h, pred)
            if float((pred - h).abs().amax()) <= tau:
                h, pred = pred, h
                taken += 1
            else:
                lbm.set_heights_device(h[0])
                lbm.step(WINDOW * (windows - w if hand_over else 1))
                lbm.get_heights_device(h[0])
                if hand_over:
                    break
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        if lbm.status() != B.MLSW_OK:
            raise RuntimeError("solver status: " + B.mlswlbm_strerror(lbm.status()))
    return h[0].cpu().numpy(), taken, secs


def lbm_rollout(params, h0, windows):
    """The same windows by the LBM alone (one solver, no restarts), timed
    like rollout(): on torch's current stream, from a synchronised start."""
    torch = _torch()
    host = np.empty((int(params["n"]), int(params["ny"]), int(params["nx"])), dtype=np.float32)
    with B.Solver(params, np.asarray(h0, dtype=np.float32),
                  stream=torch.cuda.current_stream()) as lbm:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.step(WINDOW * windows)
        lbm.get_heights(host)
        secs = time.perf_counter() - t0
    return host, secs


def film_statistics(h, hstar):
    """Largest-scale statistics of a dewetting film that do not depend on the
    exact pattern: per layer the fraction of cells below 2 h* and the
    standard deviation of the heights."""
    h = np.asarray(h, dtype=np.float64)
    return {"dewetted_fraction": [float((h[i] < 2 * hstar).mean()) for i in range(h.shape[0])],
            "height_std": [float(h[i].std()) for i in range(h.shape[0])]}


def first_rupture(traj_heights, hstar):
    """Index of the first window whose heights fall below 1.5 h* anywhere
    (None if none)."""
    for w, h in enumerate(traj_heights):
        if float(np.min(h)) < 1.5 * hstar:
            return w
    return None
