"""Learned p_det surrogate: features, training on campaign outcomes, h0 at a target p_det.

The network (ft_mlp, trained and evaluated by the library's CUDA kernels) maps
    [log10 c, log10 S_ref, duty cycle, n_x, n_y, n_z, f0 position in the band, f1 / 1e-9,
     A+^2, Ax^2, cos 4psi, sin 4psi, tau]
to the probability that the search detects the signal (Sec. V's p_det), where
c = h0 / sqrt(S_ref / T_SFT), A+ = (1 + cos^2 iota) / 2 and Ax = cos iota.  The signal power
per SFT is (F+ A+)^2 + (Fx Ax)^2 (Sec. II), and psi enters F+ and Fx through 2 psi, so the
squared amplitudes and the 4 psi harmonics are the orientation terms it depends on; given
them, detection is close to a step in c and the network learns it from few injections.
tau is the band's threshold (Sec. V.B's detection rule): it is estimated per band from
noise-only searches, and its statistical scatter between bands moves the band's 90% point,
so the network sees it rather than averaging over it.
The amplitude at which a band reaches p_det = p is the root in log10 c of the network's
p_det averaged over the signal population (sky, orientation, f0, f1) drawn as in the
campaign (Eq. (sampling)), found by bisection with BF16 inference.

Early stopping on noisy outcomes leaves a single network's 90% point a few per cent off in
either direction depending on its initialisation and validation split; the surrogate is
therefore a small ensemble whose members differ in both, and p_det is the members' mean.
"""
from __future__ import annotations

import math

import numpy as np

from . import MLP

N_FEATURES = 13


def features(log10_c, log10_s, duty, n, f0_frac, f1, cosi, psi, tau):
    """Feature matrix [n_samples, 13] (FP64; standardised and cast to FP32 by Surrogate)."""
    m = len(log10_c)
    cosi = np.asarray(cosi, np.float64)
    psi = np.asarray(psi, np.float64)
    F = np.empty((m, N_FEATURES), np.float64)
    F[:, 0] = log10_c
    F[:, 1] = log10_s
    F[:, 2] = duty
    F[:, 3:6] = n
    F[:, 6] = f0_frac
    F[:, 7] = np.asarray(f1, np.float64) / 1e-9
    F[:, 8] = (0.5 * (1.0 + cosi * cosi)) ** 2
    F[:, 9] = cosi * cosi
    F[:, 10] = np.cos(4.0 * psi)
    F[:, 11] = np.sin(4.0 * psi)
    F[:, 12] = tau
    return F


class TrainingInterrupted(RuntimeError):
    """Raised by Surrogate.fit(stop_after=...) once its pass budget is spent."""


def _load_checkpoint(path):
    import os

    if path is None or not os.path.exists(path):
        return None
    with np.load(path, allow_pickle=False) as z:
        return {k: z[k] for k in z.files}


def _save_checkpoint(path, hist, done, cur, finals=None):
    """Write the training state atomically: members 0 .. done-1 finished (their losses, best
    pass and final parameters), and the current member's state if any."""
    import os

    d = {"done": np.int64(done)}
    prev = _load_checkpoint(path) or {}
    for i in range(done):
        tr, va, be = hist[i]
        d[f"tr_{i}"], d[f"va_{i}"], d[f"best_ep_{i}"] = tr, va, np.int64(be)
        d[f"final_{i}"] = finals[i] if finals is not None else prev[f"final_{i}"]
    if cur is not None:
        for k, v in cur.items():
            d[k] = np.asarray(v)
    tmp = path + ".tmp.npz"
    np.savez(tmp, **d)
    os.replace(tmp, path)


class Surrogate:
    def __init__(self, ctx, width=128, seed=0, members=5):
        self.nets = [MLP(ctx, N_FEATURES, width, seed=seed * 7919 + i) for i in range(members)]
        self.mu = None
        self.sd = None

    def _std(self, F):
        return ((F - self.mu) / self.sd).astype(np.float32)

    def fit(self, F, y, epochs=200, batch=1024, lr=2e-3, seed=0, val_frac=0.1, patience=12,
            checkpoint=None, every=10, stop_after=None):
        """Train every member on the GPU one pass at a time on its own seeded split, keeping
        the parameters of the pass with the lowest binary cross entropy on that member's
        validation part (early stopping: the outcomes are noisy, so a long run memorises
        noise and over-states p_det).  Returns per member (training losses, validation
        losses, best pass).

        checkpoint: a file path; the training state (finished members, the current member's
        parameters, Adam moments and step count, losses and best pass) is written every
        `every` passes and when a member finishes, and a call with the same arguments
        resumes from it with results identical to an uninterrupted run.  stop_after: stop
        (raising TrainingInterrupted) after that many passes of this call, for budgets."""
        y = np.asarray(y, np.float32)
        self.mu = F.mean(0)
        self.sd = F.std(0) + 1e-12
        X = self._std(F)
        hist = []
        ck = _load_checkpoint(checkpoint)
        passes = 0
        for i, net in enumerate(self.nets):
            if ck is not None and i < ck["done"]:
                net.set_params(ck[f"final_{i}"])
                hist.append((ck[f"tr_{i}"], ck[f"va_{i}"], int(ck[f"best_ep_{i}"])))
                continue
            g = np.random.default_rng(seed * 1000 + i)
            perm = g.permutation(len(y))
            n_val = max(1, int(round(val_frac * len(y))))
            vi, ti = perm[:n_val], perm[n_val:]
            Xt, yt = X[ti], y[ti]
            Xv, yv = X[vi], y[vi].astype(np.float64)
            best, best_ep, best_theta = np.inf, -1, None
            tr, va = [], []
            ep0 = 0
            if ck is not None and i == ck["done"] and "cur_state" in ck:
                net.set_state(ck["cur_state"], int(ck["cur_t"]))
                tr, va = list(ck["cur_tr"]), list(ck["cur_va"])
                best, best_ep = float(ck["cur_best"]), int(ck["cur_best_ep"])
                best_theta = ck["cur_best_theta"]
                ep0 = len(tr)
            for ep in range(ep0, epochs):
                tr.append(float(net.train(Xt, yt, batch=batch, epochs=1, lr=lr,
                                          seed=(seed * 1000 + i) * 1000003 + ep)[0]))
                p = np.clip(net.predict(Xv, bf16=False).astype(np.float64), 1e-7, 1 - 1e-7)
                v = float(-np.mean(yv * np.log(p) + (1 - yv) * np.log(1 - p)))
                va.append(v)
                if v < best:
                    best, best_ep, best_theta = v, ep, net.get_params()
                elif ep - best_ep >= patience:
                    break
                passes += 1
                if checkpoint is not None and ep + 1 < epochs and (ep + 1) % every == 0:
                    st, t = net.get_state()
                    _save_checkpoint(checkpoint, hist, i, dict(
                        cur_state=st, cur_t=t, cur_tr=np.array(tr), cur_va=np.array(va),
                        cur_best=best, cur_best_ep=best_ep, cur_best_theta=best_theta))
                if stop_after is not None and passes >= stop_after and ep + 1 < epochs:
                    raise TrainingInterrupted(f"stopped after {passes} passes")
            net.set_params(best_theta)
            hist.append((np.array(tr), np.array(va), best_ep))
            if checkpoint is not None:
                _save_checkpoint(checkpoint, hist, i + 1, None, [n.get_params() for n in self.nets[:i + 1]])
        return hist

    def p(self, F, bf16=True):
        X = self._std(F)
        return np.mean([net.predict(X, bf16=bf16) for net in self.nets], axis=0)

    def log10_c_at(self, p, log10_s, duty, tau, pop, lo=-1.5, hi=2.5, bf16=True, iters=40):
        """Root in log10 c of mean_pop p_det = p; pop = dict(n [m,3], f0_frac, f1, cosi, psi
        [m])."""
        m = len(pop["f0_frac"])

        def mean_p(lc):
            F = features(np.full(m, lc), np.full(m, log10_s), np.full(m, duty), pop["n"],
                         pop["f0_frac"], pop["f1"], pop["cosi"], pop["psi"], np.full(m, tau))
            return float(np.mean(self.p(F, bf16=bf16)))

        a, b = lo, hi
        fa, fb = mean_p(a) - p, mean_p(b) - p
        if fa * fb > 0:
            return math.nan
        for _ in range(iters):
            mid = 0.5 * (a + b)
            fm = mean_p(mid) - p
            if (fm > 0) == (fb > 0):
                b, fb = mid, fm
            else:
                a, fa = mid, fm
        return 0.5 * (a + b)

    def close(self):
        for net in self.nets:
            net.close()
