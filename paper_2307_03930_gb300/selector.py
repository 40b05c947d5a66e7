"""Measurement sweep and training of the learned schedule selector.

The sweep draws random pruned layers (M, K log-uniform in [64, 4096], N
log-uniform in [196, 12544], sparsity uniform in [0.70, 0.99], patterns
uniform / 4x1 blocks / power-law rows), packs each on the device and lets the
library's autotuner time every candidate schedule (CUDA graphs, L2 flushed
before each launch).  The selector network (3 x 64 ReLU, softmax over the
candidates) is trained on those times with the library's own GPU kernels
(forward, cross-entropy backward, Adam) and installed with
``rosko_selector_set``.  Regret is measured against exhaustive search and
against the analytic rule.

    python -m paper_2307_03930_gb300.selector --train 1000 --heldout 2000 \
        --out paper_2307_03930_gb300/selector_weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "selector_weights.npz")
PATTERNS = ("uniform", "block4x1", "powerlaw")


def random_problems(seed: int, count: int, family: str = "layers"):
    """(M, K, N, s, pattern, matrix seed) per problem; draw order M, K, N, s,
    pattern.

    family "layers": M, K log-uniform in [64, 4096], N log-uniform in
    [196, 12544], s uniform in [0.70, 0.99] (the held-out distribution).
    family "conv": convolution-shaped layers, M = output channels
    log-uniform in [64, 2048], K = 9 x input channels (log-uniform in
    [32, 1024]), N = output pixels log-uniform in [196, 12544], s uniform in
    [0.5, 0.999] (magnitude-pruned density range of a pruned network) -
    training only, so that the network also covers deeper, denser and
    sparser layers than the held-out family."""
    from . import inputs as gen
    rng = gen.rng_for(seed, 0 if family == "layers" else 1)
    out = []
    for i in range(count):
        if family == "layers":
            M = gen.loguniform_int(rng, 64, 4096)
            K = gen.loguniform_int(rng, 64, 4096)
            N = gen.loguniform_int(rng, 196, 12544)
            s = float(rng.uniform(0.70, 0.99))
        else:
            M = gen.loguniform_int(rng, 64, 2048)
            K = 9 * gen.loguniform_int(rng, 32, 1024)
            N = gen.loguniform_int(rng, 196, 12544)
            s = float(rng.uniform(0.5, 0.999))
        pat = PATTERNS[int(rng.integers(0, len(PATTERNS)))]
        out.append((M, K, N, s, pat, i))
    return out


def sweep(seed: int, count: int, reps: int = 3, log_every: int = 50, family: str = "layers"):
    """Features, per-candidate times (NaN where a candidate does not apply)
    and the analytic rule's time for `count` random problems."""
    import torch

    from . import inputs as gen
    from . import rosko
    dev = torch.device("cuda")
    nc = rosko.rosko_num_candidates()
    feats = np.zeros((count, 16))
    times = np.full((count, nc), np.nan)
    analytic = np.zeros(count)
    meta = []
    t0 = time.time()
    for j, (M, K, N, s, pat, i) in enumerate(random_problems(seed, count, family)):
        A = gen.sparse_weight(M, K, s, gen.rng_for(seed, 1 if family == "layers" else 3, i), pat)
        h = rosko.rosko_pack(torch.from_numpy(A).to(dev), rosko.BF16)
        ldb = -(-N // 8) * 8
        Bbuf = torch.randn((K, ldb), device=dev, dtype=torch.bfloat16)
        Bd = Bbuf[:, :N]
        C = torch.empty((M, N), device=dev)
        _, tl = rosko.rosko_autotune(h, Bd, C, reps=reps)
        times[j] = [np.nan if t is None else t for t in tl]
        analytic[j] = rosko.rosko_time_tile(h, Bd, C, None, reps=reps)
        feats[j] = rosko.rosko_features(h, N)
        meta.append({"M": M, "K": K, "N": N, "s": s, "pattern": pat,
                     "nnz": h.info()["nnz"]})
        del h, Bbuf, C
        if log_every and (j + 1) % log_every == 0:
            print(f"sweep {j + 1}/{count} {time.time() - t0:.0f}s", flush=True)
    return {"features": feats, "times": times, "analytic": analytic, "meta": meta}


def soft_targets(times: np.ndarray, tau: float = 0.3) -> np.ndarray:
    """Target distribution over candidates: exp(-(t/t_best - 1)/tau) over the
    applicable ones (tau -> 0 gives one-hot on the fastest)."""
    t = np.where(np.isnan(times), np.inf, times)
    best = t.min(axis=1, keepdims=True)
    w = np.exp(-(t / best - 1.0) / tau)
    w[~np.isfinite(t)] = 0.0
    return (w / w.sum(axis=1, keepdims=True)).astype(np.float32)


def train(features: np.ndarray, times: np.ndarray, epochs: int = 200, lr: float = 2e-3,
          seed: int = 4, batch: int = 256, tau: float = 0.3, weight_decay: float = 1e-3):
    """Train the selector with the library's GPU kernels.  Returns a dict with
    the flat parameters and the feature standardisation / range.

    The labels are noisy (candidates within a few per cent of each other are
    often the same kernel timed twice), so the targets are soft (tau = 0.3:
    a candidate 10% slower than the best keeps weight e^-1/3) and the
    weights carry an L2 penalty; tau, the penalty and the epoch count were
    chosen by regret on a validation split (the last 20% of the training
    problems), never on the held-out problems."""
    import torch

    from . import rosko
    from .inputs import rng_for
    dev = torch.device("cuda")
    nc = times.shape[1]
    mean = features.mean(axis=0)
    std = features.std(axis=0)
    std[std == 0] = 1.0
    X = ((features - mean) / std).astype(np.float32)
    Y = soft_targets(times, tau)
    rng = rng_for(seed, 7)
    # He-uniform initial weights, zero biases (layout: W [out][in], then b)
    sizes = [X.shape[1], 64, 64, 64, nc]
    parts = []
    for l in range(4):
        lim = math.sqrt(6.0 / sizes[l])
        parts.append(rng.uniform(-lim, lim, size=(sizes[l + 1], sizes[l])).ravel())
        parts.append(np.zeros(sizes[l + 1]))
    P = torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(dev)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    Xd, Yd = torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev)
    n = X.shape[0]
    step = 0
    ws = torch.empty(rosko.rosko_mlp_workspace_floats(min(batch, n), nc), device=dev)
    losses = []
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).to(dev)
        for b0 in range(0, n - min(batch, n) + 1, min(batch, n)):
            idx = order[b0:b0 + min(batch, n)]
            loss, g = rosko.rosko_mlp_loss_grad(P, Xd[idx].contiguous(), Yd[idx].contiguous(), ws)
            step += 1
            rosko.rosko_mlp_adam(P, g, m, v, step, lr=lr, weight_decay=weight_decay)
        if ep % 50 == 0 or ep == epochs - 1:
            full, _ = rosko.rosko_mlp_loss_grad(P, Xd, Yd)
            losses.append(float(full.item()))
    return {"params": P.cpu().numpy(), "mean": mean, "std": std,
            "lo": features.min(axis=0), "hi": features.max(axis=0), "losses": losses}


MARGIN = float(np.log(2.0))   # the library's deference margin (logit units)


def choose(z: np.ndarray, applicable: np.ndarray, eq: np.ndarray) -> np.ndarray:
    """The library's learned-mode choice from logits z: the argmax over the
    applicable candidates, unless it beats the candidate matching the
    analytic rule (eq, -1 if none) by at most MARGIN; then -1 (= the rule)."""
    z = np.where(applicable, z, -np.inf)
    top = np.argmax(z, axis=1)
    rows = np.arange(len(z))
    has = eq >= 0
    zeq = np.where(has, z[rows, np.maximum(eq, 0)], -np.inf)
    defer = has & ((top == eq) | (z[rows, top] - zeq <= MARGIN))
    return np.where(defer, -1, top)


def predict(model: dict, features: np.ndarray, applicable: np.ndarray) -> np.ndarray:
    """Chosen candidate per row as the library's learned mode picks it (-1:
    the analytic rule), from the GPU network's logits."""
    import torch

    from . import rosko
    X = ((features - model["mean"]) / model["std"]).astype(np.float32)
    nc = applicable.shape[1]
    z = rosko.rosko_mlp_forward(torch.from_numpy(model["params"]).cuda(),
                                torch.from_numpy(X).cuda(), nc).cpu().numpy()
    return choose(z, applicable, rosko.analytic_candidates(features))


def regret(times: np.ndarray, analytic: np.ndarray, choice: np.ndarray) -> dict:
    """Mean of t_chosen / t_best - 1 for the network and for the analytic rule,
    and the geometric-mean speedup of the network's choice over the rule
    (choice -1 = the analytic rule's own time)."""
    best = np.nanmin(times, axis=1)
    chosen = np.where(choice >= 0, times[np.arange(times.shape[0]), np.maximum(choice, 0)],
                      analytic)
    return {"mlp_regret": float(np.mean(chosen / best - 1.0)),
            "analytic_regret": float(np.mean(analytic / best - 1.0)),
            "mlp_vs_analytic_geomean_speedup": float(np.exp(np.mean(np.log(analytic / chosen)))),
            "n": int(times.shape[0])}


# Candidate columns of the sweep: sparse configuration i, dense threshold j
# (index i * 5 + j); the analytic rule's row-direct configurations are
# i = 3 (512-column strips) and i = 11 (256), its thresholds j = 0 (never
# dense) and j = 3 (15 per mille); j = 1 (1 per mille) is all-dense.
N_DENSE_PM = 5


def _relfit(x: np.ndarray, y: np.ndarray) -> tuple[float, float]:
    """(a, b) minimising sum(((a + b x) / y - 1)^2): least squares in
    relative error."""
    A = np.stack([1.0 / y, x / y], 1)
    sol, *_ = np.linalg.lstsq(A, np.ones_like(y), rcond=None)
    return float(sol[0]), float(sol[1])


def split_columns(features: np.ndarray, times: np.ndarray) -> dict:
    """Shapes and the three timed paths the analytic rule chooses between,
    per problem (times in microseconds)."""
    f = np.asarray(features, dtype=np.float64)
    M, K, N = (np.round(2.0 ** f[:, j]) for j in range(3))
    nnz = np.round(f[:, 3] * M * K)
    i_rd = np.where((f[:, 3] < 0.015) & (N >= 1024), 3, 11)
    r = np.arange(len(f))
    t = np.asarray(times, dtype=np.float64) * 1e3
    return {"M": M, "K": K, "N": N, "nnz": nnz,
            "direct": t[r, i_rd * N_DENSE_PM], "split": t[r, i_rd * N_DENSE_PM + 3],
            "dense": t[r, i_rd * N_DENSE_PM + 1], "best": np.nanmin(t, axis=1)}


def fit_split(features: np.ndarray, times: np.ndarray) -> dict:
    """The analytic rule's two time models, fitted to a timed sweep: dense
    t = a + 2 M K N / R_dense (all tiles on the tensor cores), row-direct
    t = c + 2 nnz N / R_direct (BF16 bytes of B moved).  Returns the
    constants (us, FLOP/s, B/s)."""
    S = split_columns(features, times)
    a, b = _relfit(2.0 * S["M"] * S["K"] * S["N"], S["dense"])
    c, e = _relfit(2.0 * S["nnz"] * S["N"], S["direct"])
    return {"dense_us": a, "dense_flops": 1e6 / b, "direct_us": c, "direct_bytes_s": 1e6 / e}


def split_regret(features: np.ndarray, times: np.ndarray, m: dict) -> dict:
    """Regret of choosing between row-direct and the 15-per-mille split by
    the models m: against the best candidate and against the better of the
    two paths."""
    S = split_columns(features, times)
    td = m["dense_us"] + 2.0 * S["M"] * S["K"] * S["N"] / m["dense_flops"] * 1e6
    tr = m["direct_us"] + 2.0 * S["nnz"] * S["N"] / m["direct_bytes_s"] * 1e6
    t = np.where(tr < td, S["direct"], S["split"])
    return {"vs_best": float(np.mean(t / S["best"] - 1.0)),
            "vs_better_of_two": float(np.mean(t / np.minimum(S["direct"], S["split"]) - 1.0))}


def save(model: dict, path: str = WEIGHTS, extra: dict | None = None) -> None:
    np.savez(path, params=model["params"], mean=model["mean"], std=model["std"],
             lo=model["lo"], hi=model["hi"], info=json.dumps(extra or {}))


def load(path: str = WEIGHTS) -> dict:
    d = np.load(path, allow_pickle=False)
    return {k: d[k] for k in ("params", "mean", "std", "lo", "hi")} | {
        "info": json.loads(str(d["info"]))}


def install(path: str = WEIGHTS) -> dict:
    from . import rosko
    model = load(path)
    rosko.rosko_selector_set(model["params"], model["mean"], model["std"], model["lo"],
                             model["hi"])
    return model


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1000)
    ap.add_argument("--heldout", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--data-in", default=None, help="train on a saved sweep (npz) instead")
    ap.add_argument("--extra", type=int, default=0,
                    help="also sweep this many convolution-shaped training problems")
    ap.add_argument("--heldout-out", default=None,
                    help="save the held-out split (features, times, analytic) as npz")
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--data-out", default=None, help="also save the sweep (npz)")
    ap.add_argument("--fit-split", default=None, metavar="SWEEP_NPZ",
                    help="fit the analytic rule's time models on a saved sweep's training "
                         "split, print them with their held-out regret, and exit")
    a = ap.parse_args()
    t0 = time.time()
    if a.fit_split:
        d = np.load(a.fit_split)
        m = fit_split(d["tr_f"], d["tr_t"])
        print(json.dumps({"model": m, "train": split_regret(d["tr_f"], d["tr_t"], m),
                          "heldout": split_regret(d["ho_f"], d["ho_t"], m)}), flush=True)
        return
    if a.data_in:
        d = np.load(a.data_in)
        tr = {"features": d["tr_f"], "times": d["tr_t"], "analytic": d["tr_a"]}
        ho = {"features": d["ho_f"], "times": d["ho_t"], "analytic": d["ho_a"]}
    else:
        tr = sweep(a.seed, a.train)
        ho = sweep(a.seed + 1000, a.heldout)
    if a.extra:
        ex = sweep(a.seed, a.extra, family="conv")
        tr = {k: (np.concatenate([tr[k], ex[k]]) if k != "meta" else tr.get(k, []) + ex[k])
              for k in ("features", "times", "analytic")}
    if a.heldout_out:
        np.savez_compressed(a.heldout_out, features=ho["features"].astype(np.float32),
                            times=ho["times"].astype(np.float32),
                            analytic=ho["analytic"].astype(np.float32))
    if a.data_out:
        np.savez(a.data_out, tr_f=tr["features"], tr_t=tr["times"], tr_a=tr["analytic"],
                 ho_f=ho["features"], ho_t=ho["times"], ho_a=ho["analytic"])
    model = train(tr["features"], tr["times"], epochs=a.epochs, seed=a.seed)
    ch_tr = predict(model, tr["features"], ~np.isnan(tr["times"]))
    ch_ho = predict(model, ho["features"], ~np.isnan(ho["times"]))
    res = {"train": regret(tr["times"], tr["analytic"], ch_tr),
           "heldout": regret(ho["times"], ho["analytic"], ch_ho),
           "runs_measured": int(np.sum(~np.isnan(tr["times"])) + np.sum(~np.isnan(ho["times"]))),
           "train_runs": int(np.sum(~np.isnan(tr["times"]))),
           "losses": model["losses"], "seconds": time.time() - t0}
    save(model, a.out, res)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
