"""Surrogate-guided dynamic-aperture (DA) scan.

The paper lists dynamic-aperture studies and DA estimates based on machine
learning among Xsuite's applications (section "Lattice modelling and single
particle tracking").  This module is the orchestration of this project's
version of it; every computation runs in the library's kernels:

1. labels: many lattice-error seeds with uneven particle counts are tracked in
   one batched persistent launch per segment (``xt_track_batched``, CUDA graph);
2. training: the MLP (``xs_mlp``) learns survival and the normalised log loss
   turn from 6 normalised initial coordinates + 10 lattice-error descriptors;
3. calibration: on a validation seed (neither trained on nor scanned) a plain
   FP64 scan on a coarser grid sets how far inside and outside the network's
   first doubtful point the true boundary can lie: the band limits;
4. scan: for a new seed the network predicts the whole polar grid, the glue
   kernels (``xs_da_select``) hand only the band to the FP64 tracker
   (``xt_track``), ``xs_da_combine`` forms the per-ray DA and flags rays whose
   boundary touches a predicted point, which are widened and re-tracked.

The plain FP64 scan tracks every grid point and is the arbiter of the
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
                   p_lo: float = 0.2, margin: int = 500, window: int = 1500, step: int | None = None,
                   max_passes: int = 6):
    """Network over the grid, FP64 tracking of the band [r_lo - margin,
    r_lo + window] around where each ray's first loss is expected, then, on
    rays whose first loss is not confirmed by a tracked survivor just inside
    it, passes that track `step` more points next to it (inward, or on both
    sides of a loss that was only predicted), the step doubling each pass.
    Returns DA index per ray, seconds, tracked points and passes."""
    import torch
    P = xtgb.Particles.from_numpy(grid)
    Xd = torch.tensor(X, device="cuda")
    r_hat = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    da = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    widen = torch.zeros(n_rays, dtype=torch.int32, device="cuda")
    st = P.t["state"]
    step = max(1, margin // 2) if step is None else max(1, int(step))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out2 = net.forward(Xd)
    xtgb.da_select(out2, n_rays, n_r, p_lo, margin, window, st, r_hat)
    tracked = 0
    passes = 0
    while True:
        tracked += int((st == 1).sum().item())
        tracker.track(P, n_turns)
        passes += 1
        xtgb.da_combine(out2, st, n_rays, n_r, da, widen)
        if passes >= max_passes or int(widen.sum().item()) == 0:
            break
        xtgb.da_select(out2, n_rays, n_r, p_lo, step, 0, st, r_hat, widen=widen, da_prev=da)
        step *= 2
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


def band_offsets(net, seed: int, n_r: int, n_theta: int, n_turns: int, n_cells: int = 20,
                 base_mult: float = 1.5, deltas=(0,), p_lo: float = 0.2):
    """Offsets of the true DA from the network's r_lo (first point it doubts,
    by ``xs_da_select``) on every ray of one seed, in beam sigmas: a plain
    FP64 scan of the seed on n_r radii gives the DA.  Returns (offsets,
    seconds)."""
    import torch
    t0 = time.perf_counter()
    el, ref, desc = seed_ring(seed, n_cells, base_mult)
    grid, (R, th, dl), n_rays = scan_grid(el, ref, n_r, n_theta, deltas)
    tr = xtgb.Tracker(el, ref)
    da, _, _ = plain_scan(tr, grid, n_rays, n_r, n_turns)
    tr.close()
    out2 = net.forward(torch.tensor(features(R, th, dl, desc), device="cuda"))
    st = torch.empty(n_rays * n_r, dtype=torch.int32, device="cuda")
    r_lo = torch.empty(n_rays, dtype=torch.int32, device="cuda")
    xtgb.da_select(out2, n_rays, n_r, p_lo, 0, 0, st, r_lo)
    return (da - r_lo.cpu().numpy()) * (R_MAX / n_r), time.perf_counter() - t0


def calibrate_band(net, seeds, n_r: int, n_theta: int, n_turns: int, n_cells: int = 20,
                   base_mult: float = 1.5, deltas=(0,), p_lo: float = 0.2, pad_sigma: float = 0.1):
    """Band limits from validation seeds (labelled with the family but neither
    the scanned seed): the band [r_lo - margin, r_lo + window] should hold the
    first loss, so margin and window are the largest inward and outward
    offsets of the DA from r_lo over all their rays, in beam sigmas, plus
    pad_sigma.  Returns (margin_sigma, window_sigma, seconds, offsets)."""
    offs, secs = [], 0.0
    for sd in seeds:
        off, t = band_offsets(net, sd, n_r, n_theta, n_turns, n_cells, base_mult, deltas, p_lo)
        offs.append(off)
        secs += t
    off = np.concatenate(offs)
    return max(0.0, -float(off.min())) + pad_sigma, max(0.0, float(off.max())) + pad_sigma, secs, off


def _stats(off):
    return None if off is None else [float(off.min()), float(np.median(off)), float(off.max())]


def da_study(family=(13, 61), test_seeds=(60, 13, 30, 45), val_seeds=(59, 41, 20), unseen_seed=200,
             mean_count=16000, n_turns=300, n_cells=20, base_mult=1.5, epochs=16, n_r=22222, n_theta=45, deltas=(0,),
             p_lo=0.2, margin_sigma=None, window_sigma=None, pad_sigma=0.1, step_sigma=0.25,
             total_labels=None, label_sigma_delta=0.0):
    """The surrogate workflow on a family of error seeds (seeds family[0] ..
    family[1]-1): random-amplitude labels of every seed tracked together in
    one batched launch per segment, the network trained on them, the band
    limits calibrated on validation seeds of the family (unless given), then
    plain / surrogate-guided / coarse scans of the test seeds of the family.
    The network's offsets on a seed outside the family measure how far it
    generalises.  total_labels scales the per-seed counts to that total;
    label_sigma_delta draws the labels' momentum deviations (0: on momentum).
    Returns a dict of the measured quantities; `per_seed` holds one entry per
    test seed and the totals are summed over them."""
    import torch
    seeds = list(range(family[0], family[1]))
    if (any(t not in seeds for t in test_seeds) or any(v not in seeds for v in val_seeds)
            or set(test_seeds) & set(val_seeds)):
        raise ValueError("test and validation seeds must be distinct members of the family")
    rng = np.random.default_rng(I.BASE_SEED + 77)
    lo, hi = math.log10(mean_count) - 0.75, math.log10(mean_count) + 0.75
    counts = np.round(10.0 ** rng.uniform(lo, hi, len(seeds))).astype(np.int64)
    if total_labels is not None:  # the same log-uniform shape, scaled to the stated total
        counts = np.maximum(1, np.round(counts * (total_labels / counts.sum()))).astype(np.int64)
    data, t_label, label_passes = make_training_set(seeds, counts, n_turns, n_cells, base_mult,
                                                    sigma_delta=label_sigma_delta)
    net = xtgb.Surrogate(seed=7)
    hist, t_train = train(net, data, epochs=epochs)
    acc_train = accuracy(net, data)
    n_r_cal = max(n_r // 10, 64)
    t_cal, off = 0.0, None
    if margin_sigma is None or window_sigma is None:
        margin_sigma, window_sigma, t_cal, off = calibrate_band(net, val_seeds, n_r_cal, n_theta, n_turns, n_cells,
                                                                base_mult, deltas, p_lo, pad_sigma)
    off_unseen = None
    if unseen_seed is not None:
        off_unseen, _ = band_offsets(net, unseen_seed, n_r_cal, n_theta, n_turns, n_cells, base_mult, deltas, p_lo)
    dr = R_MAX / n_r
    margin, window = int(round(margin_sigma / dr)), int(round(window_sigma / dr))
    step = max(1, int(round(step_sigma / dr)))
    per_seed = []
    for ts in test_seeds:
        el, ref, desc = seed_ring(ts, n_cells, base_mult)
        grid, (R, th, dl), n_rays = scan_grid(el, ref, n_r, n_theta, deltas)
        X = features(R, th, dl, desc)
        tr = xtgb.Tracker(el, ref)
        # Run every scan once on a small grid of the same ring first: the first
        # use of a device kernel (ours or torch's) loads its module, which can
        # take seconds and must not land inside the timed scans.
        n_r_w = 256
        grid_w, (R_w, th_w, dl_w), _ = scan_grid(el, ref, n_r_w, n_theta, deltas)
        X_w = features(R_w, th_w, dl_w, desc)
        plain_scan(tr, grid_w, n_rays, n_r_w, 2)
        surrogate_scan(tr, net, grid_w, X_w, n_rays, n_r_w, 2, p_lo, 4, 8, 2)
        coarse_scan(tr, grid_w, n_rays, n_r_w, 2)
        da_p, t_plain, _ = plain_scan(tr, grid, n_rays, n_r, n_turns)
        t0 = time.perf_counter()
        net.forward(torch.tensor(X, device="cuda"))
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        da_s, t_sur, n_sur, passes = surrogate_scan(tr, net, grid, X, n_rays, n_r, n_turns, p_lo, margin, window,
                                                    step)
        da_c, t_coarse, n_coarse = coarse_scan(tr, grid, n_rays, n_r, n_turns)
        tr.close()
        err_s = np.abs(da_s - da_p) * dr
        err_c = np.abs(da_c - da_p) * dr
        per_seed.append(dict(
            seed=int(ts), labels=int(counts[seeds.index(ts)]), n_elements=int(el.shape[0]),
            da_plain_sigma_min_median_max=_stats(da_p * dr), plain_seconds=t_plain, surrogate_seconds=t_sur,
            inference_seconds=t_inf, speedup=t_plain / t_sur, tracked_fraction=n_sur / (n_rays * n_r),
            passes=passes, da_error_sigma_max=float(err_s.max()), da_error_sigma_mean=float(err_s.mean()),
            rays_within_0p2_sigma=float(np.mean(err_s <= 0.2 + 1e-9)), coarse_seconds=t_coarse,
            coarse_speedup=t_plain / t_coarse, coarse_tracked_fraction=n_coarse / (n_rays * n_r),
            coarse_da_error_sigma_max=float(err_c.max()),
            coarse_rays_within_0p2_sigma=float(np.mean(err_c <= 0.2 + 1e-9))))
    net.close()
    tp = sum(r["plain_seconds"] for r in per_seed)
    tsur = sum(r["surrogate_seconds"] for r in per_seed)
    tco = sum(r["coarse_seconds"] for r in per_seed)
    overhead = (t_label + t_train + t_cal) / len(seeds)
    return dict(
        family_seeds=len(seeds), test_seeds=[int(t) for t in test_seeds], val_seeds=[int(v) for v in val_seeds],
        n_train=int(data["X"].shape[0]), label_seconds=t_label, label_passes=label_passes, train_seconds=t_train,
        epochs=epochs, loss_history=hist, train_accuracy=acc_train,
        p_lo=p_lo, margin_sigma=float(margin_sigma), window_sigma=float(window_sigma), pad_sigma=pad_sigma,
        step_sigma=step_sigma, calibration_seconds=t_cal, calibration_offsets_sigma=_stats(off),
        unseen_seed=unseen_seed, unseen_offsets_sigma=_stats(off_unseen),
        n_turns=n_turns, grid_points=int(n_theta * len(deltas) * n_r), n_rays=int(n_theta * len(deltas)),
        n_r=int(n_r), plain_seconds_total=tp, surrogate_seconds_total=tsur, coarse_seconds_total=tco,
        speedup=tp / tsur, speedup_min=min(r["speedup"] for r in per_seed),
        speedup_max=max(r["speedup"] for r in per_seed),
        family_overhead_seconds_per_seed=overhead,
        speedup_with_overhead=tp / (tsur + overhead * len(per_seed)),
        da_error_sigma_max=max(r["da_error_sigma_max"] for r in per_seed),
        rays_within_0p2_sigma=float(np.mean([r["rays_within_0p2_sigma"] for r in per_seed])),
        max_passes_used=max(r["passes"] for r in per_seed),
        coarse_speedup=tp / tco, coarse_da_error_sigma_max=max(r["coarse_da_error_sigma_max"] for r in per_seed),
        coarse_rays_within_0p2_sigma=float(np.mean([r["coarse_rays_within_0p2_sigma"] for r in per_seed])),
        per_seed=per_seed,
    )


def da_study_full(n_turns: int = 100, base_mult: float = 1.0, total_labels: int = 5_000_000, epochs: int = 16,
                  test_seeds=(60, 13, 30, 45), val_seeds=(59, 41, 20), unseen_seed=200):
    """The surrogate workflow on the LHC-scale ring itself (200 cells,
    20,000 elements): a family of 64 error seeds with per-seed log-uniform
    scales of the orders 2..6 in [0.5, 2] (times base_mult), total_labels
    random-amplitude labels over the family with momentum deviations
    N(0, sigma_delta), and scans of the full 999,990-point grid (22,222 radii
    x 9 angles x 5 momentum offsets -2..2 sigma_delta) of the test seeds."""
    return da_study(family=(0, 64), test_seeds=test_seeds, val_seeds=val_seeds, unseen_seed=unseen_seed,
                    mean_count=total_labels / 64, n_turns=n_turns, n_cells=200, base_mult=base_mult,
                    epochs=epochs, n_r=22222, n_theta=9, deltas=(-2, -1, 0, 1, 2), total_labels=total_labels,
                    label_sigma_delta=SIGMA_DELTA)
