"""Surrogate-guided dynamic-aperture (DA) scan.

The paper lists dynamic-aperture studies and DA estimates based on machine
learning among Xsuite's applications (section "Lattice modelling and single
particle tracking").  This module is the orchestration of this project's
version of it; every computation runs in the library's kernels:

1. labels: many lattice-error seeds with uneven particle counts are tracked in
   one batched persistent launch per segment (``xt_track_batched``, CUDA graph);
2. training: the MLP (``xs_mlp``) learns survival and the normalised log loss
   turn from 6 normalised initial coordinates + 10 lattice-error descriptors;
3. scan: for a new seed the network predicts the whole polar grid, the glue
   kernels (``xs_da_select``) hand only the uncertain band to the FP64 tracker
   (``xt_track``), ``xs_da_combine`` forms the per-ray DA and flags rays whose
   boundary touches a predicted point, which are widened and re-tracked.

The plain FP64 scan tracks every grid point and is the judge of the
surrogate's DA error, stated in beam sigmas.  A non-learned baseline places the
band from a coarse FP64 grid instead.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs as I
from . import xtgb

SIGMA_DELTA = 3e-4
R_MAX = 20.0


def features(r, theta, delta, desc) -> np.ndarray:
    """16 inputs: normalised (x, px, y, py, zeta, delta) at element 0 with
    x = r cos(theta)/R_MAX, y = r sin(theta)/R_MAX (normalised momenta and zeta
    are zero on the scan grid), delta/(3 sigma_delta), and the 10 lattice-error
    descriptors log(s)/log(2)."""
    n = r.shape[0]
    X = np.zeros((n, 16), dtype=np.float32)
    X[:, 0] = r * np.cos(theta) / R_MAX
    X[:, 2] = r * np.sin(theta) / R_MAX
    X[:, 5] = delta / (3 * SIGMA_DELTA)
    X[:, 6:] = np.asarray(desc, dtype=np.float64)[None, :] / math.log(2.0)
    return X


def seed_ring(i: int, n_cells: int = 20, base_mult: float = 1.5):
    """Error seed i of the reduced LHC-scale ring: per-seed log-uniform scales of
    the normal/skew orders 2..6 (the descriptors) times a global multiplier."""
    scales, desc = I.seed_error_scales(i)
    el, ref = I.lhc_ring(seed=I.BASE_SEED + 1000 + i, n_cells=n_cells, error_scales=base_mult * scales)
    return el, ref, desc


def make_training_set(seed_ids, counts, n_turns: int, n_cells: int = 20, base_mult: float = 1.5,
                      graph: bool = True, sigma_delta: float = 0.0):
    """Tracks counts[j] random-amplitude particles of every seed for n_turns
    turns in one batched launch; returns the samples and the tracking time."""
    import torch
    trs, ps, meta = [], [], []
    for j, i in enumerate(seed_ids):
        el, ref, desc = seed_ring(i, n_cells, base_mult)
        p = I.polar_sample(el, ref, int(counts[j]), seed=I.BASE_SEED + 5000 + i, r_max=R_MAX,
                           sigma_delta=sigma_delta)
        r, th, dl = p["norm"]
        trs.append(xtgb.Tracker(el, ref))
        ps.append(xtgb.Particles.from_numpy(I.subset(p, np.arange(int(counts[j])))))
        meta.append((r, th, dl, desc, i))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xtgb.track_batched(trs, ps, n_turns, 0, graph=graph)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    Xs, ys, ts, ms, sid = [], [], [], [], []
    passes = 0
    for P, (r, th, dl, desc, i) in zip(ps, meta):
        o = P.to_numpy()
        surv = o["state"] == 1
        lost_turn = np.where(surv, n_turns, o["at_turn"]).astype(np.float64)
        n_el = trs[0].table.shape[0]
        passes += int(surv.sum()) * n_turns * n_el + int((o["at_turn"][~surv].astype(np.int64) * n_el
                                                            + o["at_element"][~surv] + 1).sum())
        Xs.append(features(r, th, dl, desc))
        ys.append(surv.astype(np.float32))
        ts.append((np.log1p(lost_turn) / math.log1p(n_turns)).astype(np.float32))
        ms.append((~surv).astype(np.float32))
        sid.append(np.full(r.shape[0], i, dtype=np.int32))
    xtgb.batched_release()
    for t in trs:
        t.close()
    data = dict(X=np.concatenate(Xs), y=np.concatenate(ys), t=np.concatenate(ts), mask=np.concatenate(ms),
                seed=np.concatenate(sid))
    return data, dt, passes


def train(net, data, epochs: int = 10, batch: int = 4096, lr: float = 1e-3, lam: float = 0.5, seed: int = 0):
    """Adam on shuffled minibatches; returns per-epoch mean loss and seconds."""
    import torch
    dev = "cuda"
    X = torch.tensor(data["X"], device=dev)
    y = torch.tensor(data["y"], device=dev)
    t = torch.tensor(data["t"], device=dev)
    m = torch.tensor(data["mask"], device=dev)
    n = X.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    hist = []
    L = torch.zeros(1, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        acc = torch.zeros(1, device=dev)
        nb = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            net.train_step(X[idx], y[idx], t[idx], m[idx], lr, lam, L)
            acc += L
            nb += 1
        hist.append(float(acc.item()) / max(nb, 1))
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def accuracy(net, data) -> float:
    import torch
    out = net.forward(torch.tensor(data["X"], device="cuda")).cpu().numpy()
    return float(np.mean((out[:, 0] >= 0) == (data["y"] > 0.5)))


# ----------------------------------------------------------------------------
def scan_grid(el, ref, n_r: int, n_theta: int = 45, deltas=(0,)):
    """Ray-major DA grid (n_rays = n_theta angles x len(deltas)) and its
    normalised coordinates.  On the reduced ring the off-momentum rays leave
    the RF bucket at once (large dispersion), so the scan is on momentum."""
    g = I.da_grid(el, ref, n_r=n_r, n_theta=n_theta, deltas=deltas, r_max=R_MAX)
    R, T, D = g["grid"]
    th = np.radians(90.0 * (T + 1) / (n_theta + 1))
    dl = np.asarray(deltas, dtype=np.float64)[D] * SIGMA_DELTA
    p = I.subset(g, np.arange(g["x"].shape[0]))
    return p, (R, th, dl), n_theta * len(deltas)


def _alive_passes(P_before_state, o, n_turns, n_el):
    st0 = P_before_state
    tracked = st0 == 1
    surv = tracked & (o["state"] == 1)
    lost = tracked & (o["state"] <= 0)
    return int(surv.sum()) * n_turns * n_el + int((o["at_turn"][lost].astype(np.int64) * n_el
                                                   + o["at_element"][lost] + 1).sum())


def plain_scan(tracker, grid: dict, n_rays: int, n_r: int, n_turns: int):
    """Tracks every grid point; DA index per ray and seconds."""
    import torch
    P = xtgb.Particles.from_numpy(grid)
    da = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tracker.track(P, n_turns)
    xtgb.da_combine(None, P.t["state"], n_rays, n_r, da)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return da.cpu().numpy(), dt, P.n


def surrogate_scan(tracker, net, grid: dict, X: np.ndarray, n_rays: int, n_r: int, n_turns: int,
                   p_lo: float = 0.02, margin: int = 500, window: int = 1500, max_passes: int = 4):
    """Network over the grid, FP64 tracking of a window around where each
    ray's first loss is expected, widened where the boundary touches a
    predicted point.  Returns DA index per ray, seconds, tracked points and
    passes."""
    import torch
    P = xtgb.Particles.from_numpy(grid)
    Xd = torch.tensor(X, device="cuda")
    r_hat = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    da = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    widen = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    st = P.t["state"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out2 = net.forward(Xd)
    xtgb.da_select(out2, n_rays, n_r, p_lo, margin, window, st, r_hat)
    tracked = 0
    passes = 0
    m = margin
    while True:
        tracked += int((st == 1).sum().item())
        tracker.track(P, n_turns)
        passes += 1
        xtgb.da_combine(out2, st, n_rays, n_r, da, widen)
        if passes >= max_passes or int(widen.sum().item()) == 0:
            break
        m *= 2
        xtgb.da_select(out2, n_rays, n_r, p_lo, m, window, st, r_hat, widen=widen, da_prev=da)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return da.cpu().numpy(), dt, tracked, passes


def coarse_scan(tracker, grid: dict, n_rays: int, n_r: int, n_turns: int, stride: int = 10):
    """Non-learned baseline: track every stride-th radius, then the radii
    between the last coarse survivor and the first coarse loss of every ray."""
    import torch
    P = xtgb.Particles.from_numpy(grid)
    st = P.t["state"]
    k = torch.arange(n_rays * n_r, device="cuda") % n_r
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    coarse = (k % stride) == (stride - 1)
    st.copy_(torch.where(coarse, 1, xtgb.XS_STATE_PREDICTED).to(torch.int32))
    tracked = int(coarse.sum().item())
    tracker.track(P, n_turns)
    S = st.view(n_rays, n_r)
    lostc = (S <= 0) & coarse.view(n_rays, n_r)
    first = torch.where(lostc.any(1), lostc.int().argmax(1), torch.full((n_rays,), n_r, device="cuda"))
    lo = (first - stride + 1).clamp(min=0)
    kk = k.view(n_rays, n_r)
    fill = (kk >= lo[:, None]) & (kk < first[:, None]) & (S == xtgb.XS_STATE_PREDICTED)
    S[S == 1] = xtgb.XS_STATE_SURVIVED
    S[fill] = 1
    tracked += int(fill.sum().item())
    tracker.track(P, n_turns)
    # untracked points count as survivors (no network output is given)
    da = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    xtgb.da_combine(None, st, n_rays, n_r, da)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return da.cpu().numpy(), dt, tracked


def da_study(train_seeds=48, test_seed=60, mean_count=4000, n_turns=1000, n_cells=20, base_mult=1.5,
             epochs=8, n_r=22222, n_theta=45, deltas=(0,), p_lo=0.02, margin_sigma=0.5, window_sigma=1.5):
    """Full study: labels, training, and plain / surrogate / coarse scans of a
    held-out seed.  Returns a dict of the measured quantities."""
    rng = np.random.default_rng(I.BASE_SEED + 77)
    lo, hi = math.log10(mean_count) - 0.75, math.log10(mean_count) + 0.75
    counts = np.round(10.0 ** rng.uniform(lo, hi, train_seeds)).astype(np.int64)
    data, t_label, label_passes = make_training_set(list(range(train_seeds)), counts, n_turns, n_cells, base_mult)
    net = xtgb.Surrogate(seed=7)
    hist, t_train = train(net, data, epochs=epochs)
    acc_train = accuracy(net, data)
    el, ref, desc = seed_ring(test_seed, n_cells, base_mult)
    grid, (R, th, dl), n_rays = scan_grid(el, ref, n_r, n_theta, deltas)
    X = features(R, th, dl, desc)
    tr = xtgb.Tracker(el, ref)
    # Run every scan once on a small grid of the same ring first: the first use
    # of a device kernel (ours or torch's) loads its module, which can take
    # seconds and must not land inside the timed scans.
    n_r_w = 256
    grid_w, (R_w, th_w, dl_w), _ = scan_grid(el, ref, n_r_w, n_theta, deltas)
    X_w = features(R_w, th_w, dl_w, desc)
    plain_scan(tr, grid_w, n_rays, n_r_w, 2)
    surrogate_scan(tr, net, grid_w, X_w, n_rays, n_r_w, 2, p_lo, 4, 8)
    coarse_scan(tr, grid_w, n_rays, n_r_w, 2)
    da_p, t_plain, n_plain = plain_scan(tr, grid, n_rays, n_r, n_turns)
    dr = R_MAX / n_r
    t0 = time.perf_counter()
    net.forward(__import__("torch").tensor(X, device="cuda"))
    __import__("torch").cuda.synchronize()
    t_inf = time.perf_counter() - t0
    da_s, t_sur, n_sur, passes = surrogate_scan(tr, net, grid, X, n_rays, n_r, n_turns, p_lo,
                                                int(round(margin_sigma / dr)), int(round(window_sigma / dr)))
    da_c, t_coarse, n_coarse = coarse_scan(tr, grid, n_rays, n_r, n_turns)
    err_s = np.abs(da_s - da_p) * dr
    err_c = np.abs(da_c - da_p) * dr
    net.close()
    tr.close()
    return dict(
        n_train=int(data["X"].shape[0]), train_seeds=int(train_seeds), label_seconds=t_label,
        label_passes=label_passes, train_seconds=t_train, epochs=epochs, loss_history=hist,
        train_accuracy=acc_train, n_turns=n_turns, n_elements=int(el.shape[0]), grid_points=int(n_rays * n_r),
        n_rays=int(n_rays), n_r=int(n_r), plain_seconds=t_plain, surrogate_seconds=t_sur,
        coarse_seconds=t_coarse, inference_seconds=t_inf, speedup=t_plain / t_sur, coarse_speedup=t_plain / t_coarse,
        tracked_fraction=n_sur / (n_rays * n_r), coarse_tracked_fraction=n_coarse / (n_rays * n_r),
        passes=passes, da_plain_sigma=(da_p * dr).tolist(),
        da_error_sigma_max=float(err_s.max()), da_error_sigma_mean=float(err_s.mean()),
        rays_within_0p2_sigma=float(np.mean(err_s <= 0.2 + 1e-9)),
        coarse_da_error_sigma_max=float(err_c.max()),
    )
