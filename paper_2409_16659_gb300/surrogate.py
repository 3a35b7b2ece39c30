"""Training and use of the U-Net surrogate of 64 LBM steps.

The network itself (mlswlbm_unet_*, BF16 kernels on the 5th-generation
tensor cores) lives in the C library; this module feeds it:

* trajectories: the heights of many instances of one lattice after every
  window of 64 steps, run by one batch of the solver, kept on the device;
* training: Adam on minibatches of (h(t), h(t + 64)) pairs drawn from
  trajectories streamed through in chunks;
* evaluation: the largest height error of each window against the LBM, next
  to that of the identity map (no change);
* the judged rollout: many instances advanced window by window by the
  surrogate, with the LBM running audit windows from the same heights; an
  instance whose audited error exceeds the bound goes back to its last
  passed audit and finishes on the LBM;
* the two plain LBM baselines of the same windows: the batched solver and
  one solver per instance.

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


def trajectories_device(params, heights, windows, stream=None):
    """Heights after 0..windows windows of every instance (all of one shape),
    read from one batch of the solver on the device: a tensor
    [instances][windows + 1][n][ny][nx]."""
    torch = _torch()
    p0 = params[0]
    n, ny, nx = int(p0["n"]), int(p0["ny"]), int(p0["nx"])
    out = torch.empty((len(params), windows + 1, n, ny, nx), dtype=torch.float32, device="cuda")
    with B.Batch(params, heights, stream=stream) as b:
        for w in range(windows + 1):
            if w:
                b.step(WINDOW)
            for j in range(len(params)):
                b.get_heights_device(j, out[j, w])
        if b.status() != B.MLSW_OK:
            raise RuntimeError("solver status: " + B.mlswlbm_strerror(b.status()))
    return out


class TrajectoryStream:
    """One batch of the solver re-used for chunk after chunk of trajectories
    of one lattice: each call restarts the instances at rest from the given
    device heights [count][n][ny][nx] and returns their heights after 0..
    windows windows, [count][windows + 1][n][ny][nx] on the device."""

    def __init__(self, params, h_first, windows, stream=None):
        self.count, self.windows = len(params), int(windows)
        self.b = B.Batch(params, [x for x in h_first.cpu().numpy()], stream=stream)

    def __call__(self, h0):
        torch = _torch()
        out = torch.empty((self.count, self.windows + 1) + tuple(h0.shape[1:]),
                          dtype=torch.float32, device="cuda")
        for j in range(self.count):
            self.b.set_heights_device(j, h0[j])
        for w in range(self.windows + 1):
            if w:
                self.b.step(WINDOW)
            for j in range(self.count):
                self.b.get_heights_device(j, out[j, w])
        return out

    def close(self):
        if self.b is not None:
            status = self.b.status()
            self.b.close()
            self.b = None
            if status != B.MLSW_OK:
                raise RuntimeError("solver status: " + B.mlswlbm_strerror(status))


def train_streaming(u, make_chunk, chunks, steps_per_chunk, batch, lr, lr_end=None, seed=0):
    """Adam steps on (h(t), h(t + 64)) pairs of trajectory chunks made one at
    a time by make_chunk(k) ([instances][windows + 1][n][ny][nx] on the
    device) and dropped after their steps; the learning rate decays
    geometrically from lr to lr_end over all steps. Returns the losses."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    lr_end = lr if lr_end is None else lr_end
    total = max(chunks * steps_per_chunk - 1, 1)
    losses, it = [], 0
    for k in range(chunks):
        traj = make_chunk(k)
        ninst, nwin = traj.shape[0], traj.shape[1] - 1
        for _ in range(steps_per_chunk):
            ii = torch.as_tensor(rng.integers(0, ninst, batch), device="cuda")
            ww = torch.as_tensor(rng.integers(0, nwin, batch), device="cuda")
            rate = lr * (lr_end / lr) ** (it / total)
            losses.append(u.train_step(traj[ii, ww].contiguous(), traj[ii, ww + 1].contiguous(),
                                       rate))
            it += 1
        del traj
    return np.array(losses)


def unet_window_errors(u, traj):
    """Per (instance, window): the U-Net's largest height error against the
    LBM, the identity map's (the window's own largest change). Arrays
    [instances][windows]."""
    torch = _torch()
    ninst, nwin = traj.shape[0], traj.shape[1] - 1
    h_all = traj[:, :-1].reshape((-1,) + tuple(traj.shape[2:]))
    t_all = traj[:, 1:].reshape((-1,) + tuple(traj.shape[2:]))
    err = []
    for k in range(0, h_all.shape[0], u.max_batch):
        h = h_all[k:k + u.max_batch].contiguous()
        pred = torch.empty_like(h)
        u.predict(h, pred)
        err.append(B.max_abs_diff(pred, t_all[k:k + u.max_batch].contiguous()))
    ident = B.max_abs_diff(t_all.contiguous(), h_all.contiguous())
    return (torch.cat(err).cpu().numpy().reshape(ninst, nwin),
            ident.cpu().numpy().reshape(ninst, nwin))


def _predict_all(u, h, out):
    for k in range(0, h.shape[0], u.max_batch):
        u.predict(h[k:k + u.max_batch].contiguous(), out[k:k + u.max_batch])
    return out


def judged_rollout(u, params, heights, windows, audit_every, bound=1e-3, stream=None):
    """Advances every instance by `windows` windows of 64 steps, by the U-Net
    (all instances in batched calls), judged by the LBM: the first window,
    every audit_every-th and the last are audits, in which the batched
    solver runs the same window from the same heights, and the largest
    height difference is the window's error. A window within `bound`
    continues from the solver's heights; an instance whose error exceeds it
    leaves the surrogate, goes back to its last passed audit and finishes on
    the LBM alone. The audits step only the instances still on the
    surrogate (mlswlbm_batch_select), and the instances that left finish in
    the same batched solver, restarted at rest from their checkpoints, in
    stages by checkpoint window so that each steps exactly its remaining
    windows. Returns (final heights [instances][n][ny][nx] tensor, a dict of
    counts, audited errors and seconds)."""
    torch = _torch()
    st = torch.cuda.current_stream() if stream is None else stream
    M = len(params)
    h = torch.stack([torch.from_numpy(np.asarray(x, dtype=np.float32)) for x in heights]).cuda()
    ckpt = h.clone()
    ckpt_w = [0] * M
    active = list(range(M))          # instances still on the surrogate
    fallback, audited = {}, []
    taken = [0] * M                  # windows taken from the surrogate since the last audit
    surrogate_windows = 0
    with B.Batch(params, [np.asarray(x, dtype=np.float32) for x in heights], stream=st) as aud:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for w in range(windows):
            if not active:
                break
            idx = torch.as_tensor(active, device="cuda")
            sub = h[idx].contiguous()
            out = torch.empty_like(sub)
            _predict_all(u, sub, out)
            if w == 0 or (w + 1) % audit_every == 0 or w == windows - 1:
                aud.set_heights_device_many(active, sub)
                aud.step(WINDOW)
                ref = torch.empty_like(sub)
                aud.get_heights_device_many(active, ref)
                err = B.max_abs_diff(out, ref, stream=st).cpu().numpy()
                audited.extend(float(e) for e in err)
                keep, keep_j = [], []
                for j, i in enumerate(active):
                    if err[j] <= bound:
                        ckpt_w[i] = w + 1
                        surrogate_windows += taken[i]
                        keep.append(i)
                        keep_j.append(j)
                    else:
                        fallback[i] = ckpt_w[i]
                    taken[i] = 0
                if keep:
                    ki = torch.as_tensor(keep, device="cuda")
                    kj = torch.as_tensor(keep_j, device="cuda")
                    h[ki] = ref[kj]
                    ckpt[ki] = ref[kj]
                if len(keep) != len(active):
                    aud.select(keep)
                active = keep
            else:
                h[idx] = out
                for i in active:
                    taken[i] += 1
        # instances that left finish on the LBM from their last passed audit
        # (the last window is always audited), all in the batch: the ones
        # with the earliest checkpoint start, the others join as the run
        # reaches their checkpoint window
        stages = sorted(set(fallback.values()))
        running = []
        for k, w0 in enumerate(stages):
            join = [i for i, wi in fallback.items() if wi == w0]
            aud.set_heights_device_many(join, ckpt[torch.as_tensor(join, device="cuda")].contiguous())
            running += join
            aud.select(running)
            w1 = stages[k + 1] if k + 1 < len(stages) else windows
            aud.step(WINDOW * (w1 - w0))
        if running:
            fin = torch.empty((len(running),) + tuple(h.shape[1:]), dtype=h.dtype, device="cuda")
            aud.get_heights_device_many(running, fin)
            h[torch.as_tensor(running, device="cuda")] = fin
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        status = aud.status()
    if status != B.MLSW_OK:
        raise RuntimeError("solver status: " + B.mlswlbm_strerror(status))
    return h, {"seconds": secs, "fallback_instances": len(fallback),
               "surrogate_windows": surrogate_windows, "audited_windows": len(audited),
               "audit_errors": audited}


def lbm_batched(params, heights, windows, stream=None):
    """The same windows by the batched solver alone; (heights tensor, seconds)."""
    torch = _torch()
    st = torch.cuda.current_stream() if stream is None else stream
    out = torch.empty((len(params),) + np.asarray(heights[0]).shape, dtype=torch.float32,
                      device="cuda")
    with B.Batch(params, [np.asarray(x, dtype=np.float32) for x in heights], stream=st) as b:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(WINDOW * windows)
        for j in range(len(params)):
            b.get_heights_device(j, out[j])
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
    return out, secs


def lbm_per_instance(params, heights, windows, stream=None):
    """The same windows by one solver per instance, stepped in turn;
    (heights tensor, seconds)."""
    torch = _torch()
    st = torch.cuda.current_stream() if stream is None else stream
    out = torch.empty((len(params),) + np.asarray(heights[0]).shape, dtype=torch.float32,
                      device="cuda")
    solvers = [B.Solver(p, np.asarray(x, dtype=np.float32), stream=st)
               for p, x in zip(params, heights)]
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in solvers:
            s.step(WINDOW * windows)
        for j, s in enumerate(solvers):
            s.get_heights_device(out[j])
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
    finally:
        for s in solvers:
            s.close()
    return out, secs
