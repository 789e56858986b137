"""The learned precision selector of the packed batch: labels from runs of the method itself,
training on the GPU with the library's own network kernels (tls_mlp_grad / tls_mlp_adam), and
the model file that tls_batch_factor(..., TLS_AUTO) uses.

Labels (per problem, "the plain method judging its error"): the batch is solved with the plain
FP64 method (u_f = u = FP64) as the reference, and with u_f in {FP16, BF16, FP32} (u = FP32,
no fallback). A run succeeds when it matches the reference to sigma rel 1e-10 and x rel 1e-8.
Its cost is a time model of the work it did: the Gram at the rate of the factor precision (the
tensor cores for FP16 / BF16, CUDA cores for FP32) plus the residual passes (FP64) and the
PCGTLS passes (FP32) it ran. The class label is the cheapest successful precision (FP32 when
none succeeds: the solve will fall back to FP64). The tolerance label is log10 of the largest
inner tolerance in {1e-1, ..., 1e-4} with which the labelled precision still succeeds in the
tolerance mode of PCGTLS (mask 0 when none does).

Features are the 16 the library computes after an FP16 factorisation (tls_batch_features).
All arithmetic of the network runs in the library's kernels; this module only moves arrays.
"""
from __future__ import annotations

import argparse
import ctypes as C
import os
import time

import numpy as np

from . import synth, tls

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_model.npz")
CLASSES = ("fp16", "bf16", "fp32")
TOLS = (1e-1, 1e-2, 1e-3, 1e-4)
SIGMA_TOL, X_TOL = 1e-10, 1e-8
# time model of a run (seconds): Gram m n^2 flops at the factor precision's rate, n^3/3 for the
# factorisation, 4 m n FP64 flops per residual pass, 4 m n bytes per FP32 pass
RATE = {"gram_tc": 1.0e15, "gram_fp32": 6.0e13, "chol": 2.0e12, "fp64": 6.0e11, "hbm": 5.0e12}


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases (flat layout W1, b1, W2, b2, W3, b3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for rows, cols in ((64, 16), (64, 64), (4, 64)):
        lim = np.sqrt(6.0 / cols)
        parts.append(rng.uniform(-lim, lim, size=rows * cols))
        parts.append(np.zeros(rows))
    return np.concatenate(parts).astype(np.float32)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class Trainer:
    """Adam on the network's FP32 master parameters, all steps in the library's kernels."""

    def __init__(self, params: np.ndarray, device: str = "cuda"):
        import torch
        self.torch = torch
        self.P = torch.tensor(params, dtype=torch.float32, device=device)
        self.m = torch.zeros_like(self.P)
        self.v = torch.zeros_like(self.P)
        self.g = torch.zeros_like(self.P)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.t = 0
        self.scratch = None

    def _check_X(self, fn: str, X) -> int:
        """X: float32 (rows, 16) contiguous on the current CUDA device; returns rows."""
        tls._check_device_tensors(fn, {"X": X}, self.torch.float32)
        if X.dim() != 2 or X.shape[1] != tls.N_FEATURES or not X.is_contiguous():
            tls._arg_error(fn, f"X must be contiguous (rows, {tls.N_FEATURES}), got "
                               f"{tuple(X.shape)}")
        return int(X.shape[0])

    def grad(self, X, ycls, ytol, ymask, idx=None, lam: float = 0.1):
        """Mean loss and gradient over the rows idx of X (all rows when idx is None). Every
        tensor is checked first (dtype, device, shape, index and label ranges): the kernel reads
        them by device pointer."""
        torch = self.torch
        fn = "tls_mlp_grad"
        rows = self._check_X(fn, X)
        tls._check_device_tensors(fn, {"ycls": ycls}, torch.int32)
        tls._check_device_tensors(fn, {"ytol": ytol, "ymask": ymask}, torch.float32)
        for nm, t in (("ycls", ycls), ("ytol", ytol), ("ymask", ymask)):
            if not t.is_contiguous() or t.numel() != rows:
                tls._arg_error(fn, f"{nm} must be contiguous with {rows} entries")
        if rows and (int(ycls.min()) < 0 or int(ycls.max()) > 2):
            tls._arg_error(fn, "ycls must hold class indices 0, 1 or 2")
        if idx is not None:
            tls._check_device_tensors(fn, {"idx": idx}, torch.int32)
            if idx.dim() != 1 or not idx.is_contiguous():
                tls._arg_error(fn, "idx must be a contiguous 1-D tensor")
            if idx.numel() and (int(idx.min()) < 0 or int(idx.max()) >= rows):
                tls._arg_error(fn, f"idx must index the {rows} rows of X")
        n = int(idx.numel()) if idx is not None else rows
        if n < 1:
            tls._arg_error(fn, "no samples")
        need = n * (tls.MLP_PARAMS + 1)
        if self.scratch is None or self.scratch.numel() < need:
            self.scratch = torch.empty(need, dtype=torch.float32, device=self.P.device)
        st = torch.cuda.current_stream().cuda_stream
        r = tls.load().tls_mlp_grad(_ptr(self.P), n, _ptr(X), _ptr(idx) if idx is not None else None,
                                    _ptr(ycls), _ptr(ytol), _ptr(ymask), C.c_float(lam),
                                    _ptr(self.scratch), _ptr(self.g), _ptr(self.loss),
                                    C.c_void_p(st))
        if r != 0:
            raise tls.TLSError(r, "tls_mlp_grad")

    def step(self, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.t += 1
        st = self.torch.cuda.current_stream().cuda_stream
        r = tls.load().tls_mlp_adam(_ptr(self.P), _ptr(self.g), _ptr(self.m), _ptr(self.v), self.t,
                                    C.c_float(lr), C.c_float(b1), C.c_float(b2), C.c_float(eps),
                                    C.c_void_p(st))
        if r != 0:
            raise tls.TLSError(r, "tls_mlp_adam")

    def forward(self, X):
        self._check_X("tls_mlp_forward", X)
        out = self.torch.empty((X.shape[0], 4), dtype=self.torch.float32, device=self.P.device)
        st = self.torch.cuda.current_stream().cuda_stream
        r = tls.load().tls_mlp_forward(_ptr(self.P), int(X.shape[0]), _ptr(X), _ptr(out),
                                       C.c_void_p(st))
        if r != 0:
            raise tls.TLSError(r, "tls_mlp_forward")
        return out

    def params(self) -> np.ndarray:
        return self.P.detach().cpu().numpy()


def normalisation(F: np.ndarray):
    mean = F.mean(axis=0).astype(np.float32)
    scale = F.std(axis=0).astype(np.float32)
    scale[scale < 1e-6] = 1.0
    return mean, scale


def train(F, ycls, ytol, ymask, epochs: int = 400, batch: int = 256, lr: float = 3e-3,
          lam: float = 0.1, seed: int = 0, params=None):
    """Minibatch Adam on the GPU. Returns (params, mean, scale, loss history)."""
    import torch
    mean, scale = normalisation(F)
    Xn = torch.tensor((F - mean) / scale, dtype=torch.float32, device="cuda")
    yc = torch.tensor(ycls, dtype=torch.int32, device="cuda")
    yt = torch.tensor(ytol, dtype=torch.float32, device="cuda")
    ym = torch.tensor(ymask, dtype=torch.float32, device="cuda")
    tr = Trainer(init_params(seed) if params is None else params)
    rng = np.random.Generator(np.random.PCG64(seed))
    n = F.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n).astype(np.int32), device="cuda")
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            tr.grad(Xn, yc, yt, ym, idx=idx, lam=lam)
            tr.step(lr)
        hist.append(float(tr.loss.item()))
    return tr.params(), mean, scale, hist


def predict(params, mean, scale, F):
    """Network outputs (n x 4) for raw features F, by the library's forward kernel."""
    import torch
    tr = Trainer(params)
    X = torch.tensor((F - mean) / scale, dtype=torch.float32, device="cuda")
    return tr.forward(X).cpu().numpy()


def _run(problems, u_f, u="fp32", **opt):
    with tls.Batch([(p.A, p.b) for p in problems]) as bt:
        bt.factor(u_f, u=u, fallback=0, **opt)
        xs, sig, infos, _ = bt.solve(tol=0.0, max_rqi=12)
        F = bt.features() if u_f == "fp16" and not opt else None
    return xs, sig, infos, F


def _cost(p, info, u_f) -> float:
    m, n = p.A.shape
    rate = RATE["gram_tc"] if u_f in ("fp16", "bf16") else RATE["gram_fp32"]
    t = m * n * n / rate + n ** 3 / 3.0 / RATE["chol"]
    t += info["rqi_steps"] * 4.0 * m * n / RATE["fp64"]
    t += (info["cg_iters"] / 2.0 + 12) * 4.0 * m * n / RATE["hbm"]
    return t


def label(problems):
    """(features, class labels, tolerance labels, tolerance mask, per-class cost, success)."""
    xr, sr, ir, _ = _run(problems, "fp64", u="fp64")
    ref_ok = np.array([i["stop_reason"] != tls.STOP_MAX_RQI for i in ir])
    k = len(problems)
    ok = np.zeros((k, 3), dtype=bool)
    cost = np.full((k, 3), np.inf)
    F = None
    for c, uf in enumerate(CLASSES):
        xs, sig, infos, F_c = _run(problems, uf)
        if F_c is not None:
            F = F_c
        for i, (p, x, s, info) in enumerate(zip(problems, xs, sig, infos)):
            good = (abs(s - sr[i]) <= SIGMA_TOL * sr[i] and
                    np.linalg.norm(x - xr[i]) <= X_TOL * np.linalg.norm(xr[i]))
            ok[i, c] = good
            if good:
                cost[i, c] = _cost(p, info, uf)
    ycls = np.where(ok.any(axis=1), np.argmin(cost, axis=1), 2).astype(np.int32)
    ytol = np.zeros(k, dtype=np.float32)
    ymask = np.zeros(k, dtype=np.float32)
    for c, uf in enumerate(CLASSES):
        sel = [i for i in range(k) if ycls[i] == c and ok[i, c]]
        if not sel:
            continue
        sub = [problems[i] for i in sel]
        best = {i: None for i in sel}
        for tol in TOLS:    # largest tolerance first
            xs, sig, infos, _ = _run(sub, uf, cg_fixed=0, cg_tol=tol, cg_max=60)
            for j, i in enumerate(sel):
                if best[i] is not None:
                    continue
                if (abs(sig[j] - sr[i]) <= SIGMA_TOL * sr[i] and
                        np.linalg.norm(xs[j] - xr[i]) <= X_TOL * np.linalg.norm(xr[i])):
                    best[i] = tol
        for i in sel:
            if best[i] is not None:
                ytol[i] = np.log10(best[i])
                ymask[i] = 1.0
    keep = ref_ok
    return F[keep], ycls[keep], ytol[keep], ymask[keep], cost[keep], ok[keep]


# ---------------------------------------------------------------------------------------------
# The wider configuration (dense and sparse problems, n up to 2048): one context per problem
# ---------------------------------------------------------------------------------------------
def _ctx(p):
    if isinstance(p, synth.CsrProblem):
        return tls.tls_create_csr(p.m, p.n, p.row_ptr, p.col_idx, p.val, p.b)
    return tls.tls_create_dense(p.A, p.b)


def _cost_any(p, info, u_f) -> float:
    """The time model of _cost for a dense problem; for CSR the Gram costs nnz * (nnz/m)^2
    FMA on CUDA cores and a pass moves the values and indices (12 bytes per entry)."""
    if not isinstance(p, synth.CsrProblem):
        return _cost(p, info, u_f)
    m, n, nnz = p.m, p.n, p.nnz
    t = 2.0 * nnz * (nnz / m) ** 2 / RATE["gram_fp32"] + n ** 3 / 3.0 / RATE["chol"]
    t += info["rqi_steps"] * 4.0 * nnz / RATE["fp64"]
    t += (info["cg_iters"] / 2.0 + 12) * 2.0 * 12.0 * nnz / RATE["hbm"]
    return t


def _close(x, s, xr, sr) -> bool:
    return bool(abs(s - sr) <= SIGMA_TOL * sr and np.linalg.norm(x - xr) <= X_TOL * np.linalg.norm(xr))


def label_one(p):
    """Labels of one problem from single-context solves on one resident copy of A: features of
    the FP16 factor, the class (cheapest precision whose own factor, not an escalated one,
    matches the plain FP64 reference), the tolerance label, per-class costs and successes, and
    whether the reference converged."""
    ctx = _ctx(p)
    try:
        tls.tls_factor(ctx, "fp64", tls.tls_default_options(u="fp64", fallback=0))
        xr, sr, ir = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
        ref_ok = ir["stop_reason"] != tls.STOP_MAX_RQI
        ok = np.zeros(3, dtype=bool)
        cost = np.full(3, np.inf)
        F = None
        for c, uf in enumerate(CLASSES):
            try:
                tls.tls_factor(ctx, uf, tls.tls_default_options(u="fp32", fallback=0))
            except tls.TLSError:
                continue
            if uf == "fp16":
                F = tls.tls_features(ctx)
            x, s, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
            if info["u_f_used"] == tls.PREC[uf] and _close(x, s, xr, sr):
                ok[c] = True
                cost[c] = _cost_any(p, info, uf)
        ycls = int(np.argmin(cost)) if ok.any() else 2
        ytol, ymask = 0.0, 0.0
        if ok[ycls]:
            for tol in TOLS:    # largest tolerance first
                tls.tls_factor(ctx, CLASSES[ycls], tls.tls_default_options(
                    u="fp32", fallback=0, cg_fixed=0, cg_tol=tol, cg_max=60))
                x, s, _ = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
                if _close(x, s, xr, sr):
                    ytol, ymask = float(np.log10(tol)), 1.0
                    break
    finally:
        tls.tls_destroy(ctx)
    return F, ycls, ytol, ymask, cost, ok, ref_ok


def dataset_wide(seed0: int, count: int, workers: int = 6, log_every: int = 500):
    """Labels of `count` problems of synth.selector_problem_wide (seeds seed0 ..), generated and
    solved by `workers` host threads, each on its own context and stream."""
    import concurrent.futures as cf

    def job(seed):
        return label_one(synth.selector_problem_wide(seed))

    rows = []
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for k, r in enumerate(ex.map(job, range(seed0, seed0 + count))):
            rows.append(r)
            if log_every and (k + 1) % log_every == 0:
                print(f"  labelled {k + 1}/{count} ({time.perf_counter() - t0:.0f} s)", flush=True)
    keep = [r for r in rows if r[6] and r[0] is not None]
    F = np.stack([r[0] for r in keep]).astype(np.float32)
    ycls = np.array([r[1] for r in keep], dtype=np.int32)
    ytol = np.array([r[2] for r in keep], dtype=np.float32)
    ymask = np.array([r[3] for r in keep], dtype=np.float32)
    cost = np.stack([r[4] for r in keep])
    ok = np.stack([r[5] for r in keep])
    return F, ycls, ytol, ymask, cost, ok


def dataset(seed0: int, count: int, chunk: int = 400):
    parts = []
    for c0 in range(0, count, chunk):
        probs = [synth.selector_problem(seed0 + i) for i in range(c0, min(count, c0 + chunk))]
        parts.append(label(probs))
    return tuple(np.concatenate([p[j] for p in parts]) for j in range(6))


def save(path, params, mean, scale, **meta):
    np.savez(path, params=np.asarray(params, dtype=np.float32), mean=mean, scale=scale, **meta)


def load_model(path: str = MODEL_PATH):
    if not os.path.exists(path):
        return None
    z = np.load(path)
    return z["params"], z["mean"], z["scale"]


def evaluate_wide(params, mean, scale, seed0: int, count: int, workers: int = 6):
    """Held-out comparison on the wider distribution, one problem at a time (so the timings are
    not shared with other solves): the plain FP64 reference, then FP16 first with the precision
    fallback, then the selector (TLS_AUTO) with the fallback. Returns per-problem arrays
    (reference converged, accurate fp16-first, accurate selector, seconds fp16-first, seconds
    selector, u_f used by the selector). Problems are generated ahead by `workers` threads."""
    import concurrent.futures as cf
    rows = []
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for p in ex.map(synth.selector_problem_wide, range(seed0, seed0 + count)):
            ctx = _ctx(p)
            try:
                tls.tls_factor(ctx, "fp64", tls.tls_default_options(u="fp64", fallback=0))
                xr, sr, ir = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
                ref_ok = ir["stop_reason"] != tls.STOP_MAX_RQI
                o = tls.tls_default_options(u="fp32")
                t0 = time.perf_counter()
                tls.tls_factor(ctx, "fp16", o)
                x1, s1, _ = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
                t1 = time.perf_counter()
                tls.tls_set_selector(ctx, params, mean, scale)
                t2 = time.perf_counter()
                tls.tls_factor(ctx, "auto", o)
                x2, s2, i2 = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
                t3 = time.perf_counter()
            finally:
                tls.tls_destroy(ctx)
            rows.append((ref_ok, _close(x1, s1, xr, sr), _close(x2, s2, xr, sr), t1 - t0, t3 - t2,
                         i2["u_f_used"]))
    return tuple(np.array([r[k] for r in rows]) for k in range(6))


def main():
    ap = argparse.ArgumentParser(description="label, train and evaluate the precision selector")
    ap.add_argument("--n-train", type=int, default=4000)
    ap.add_argument("--n-eval", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--wide", action="store_true",
                    help="the wider distribution (dense and sparse, n up to 2048), one context per "
                         "problem; seeds 200000.. training, 300000.. held out")
    ap.add_argument("--workers", type=int, default=6)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    if args.wide:
        main_wide(args)
        return
    t0 = time.time()
    Ftr, ytr, ttr, mtr, ctr, oktr = dataset(10000, args.n_train)
    Fev, yev, tev, mev, cev, okev = dataset(100000, args.n_eval)
    t1 = time.time()
    params, mean, scale, hist = train(Ftr, ytr, ttr, mtr, epochs=args.epochs)
    t2 = time.time()
    out = predict(params, mean, scale, Fev)
    pred = out[:, :3].argmax(axis=1)
    acc = float((pred == yev).mean())
    # cost of the chosen precision on held-out problems vs FP16 first (with fallback: a failed
    # FP16 run is paid for and then the labelled precision's run)
    fb = np.where(okev[:, 0], cev[:, 0], np.nan)
    print(f"labels {t1 - t0:.1f}s train {t2 - t1:.1f}s; train {len(ytr)} eval {len(yev)}; "
          f"class mix train {np.bincount(ytr, minlength=3).tolist()} eval "
          f"{np.bincount(yev, minlength=3).tolist()}; eval accuracy {acc:.3f}; "
          f"final loss {hist[-1]:.4f}; FP16 success rate {okev[:, 0].mean():.3f}", flush=True)
    save(args.out, params, mean, scale, loss=np.array(hist), eval_accuracy=acc,
         n_train=len(ytr), n_eval=len(yev))


def main_wide(args):
    t0 = time.time()
    Ftr, ytr, ttr, mtr, ctr, oktr = dataset_wide(200000, args.n_train, workers=args.workers)
    Fev, yev, tev, mev, cev, okev = dataset_wide(300000, args.n_eval, workers=args.workers)
    t1 = time.time()
    params, mean, scale, hist = train(Ftr, ytr, ttr, mtr, epochs=args.epochs)
    t2 = time.time()
    out = predict(params, mean, scale, Fev)
    acc = float((out[:, :3].argmax(axis=1) == yev).mean())
    print(f"labels {t1 - t0:.1f}s train {t2 - t1:.1f}s; train {len(ytr)} eval {len(yev)}; "
          f"class mix train {np.bincount(ytr, minlength=3).tolist()} eval "
          f"{np.bincount(yev, minlength=3).tolist()}; eval accuracy {acc:.3f}; "
          f"final loss {hist[-1]:.4f}", flush=True)
    ref_ok, ok1, ok2, sec1, sec2, uf2 = evaluate_wide(params, mean, scale, 300000,
                                                      args.n_eval, workers=args.workers)
    sel = ref_ok.astype(bool)
    res = {"eval_problems": int(sel.sum()), "accurate_fp16_first": int(ok1[sel].sum()),
           "accurate_selector": int(ok2[sel].sum()), "seconds_fp16_first": float(sec1[sel].sum()),
           "seconds_selector": float(sec2[sel].sum()),
           "selector_u_f_hist": np.bincount(uf2[sel].astype(int), minlength=4).tolist()}
    print("held-out:", res, flush=True)
    save(args.out, params, mean, scale, loss=np.array(hist), eval_accuracy=acc,
         n_train=len(ytr), n_eval=len(yev), **{k: np.array(v) for k, v in res.items()})


if __name__ == "__main__":
    main()
