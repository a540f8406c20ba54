"""CPU oracle of the IG host helpers -- TEST INFRASTRUCTURE ONLY.

Plain Python statements of the preprocessing and evaluation around IG, used
to check the library's host helpers.  Like the rest of ``oracle/`` it may be
imported only by the tests, ``__graft_entry__.smoke()`` and the CPU baseline
leg of ``bench.py``, and it shares no code with the library.

* ``discretize``: Section 3.1 -- numeric attributes are z-scored and rounded
  to p decimals, categorical values are taken as they are, and each (column,
  value) pair is one token.  Readings (the paper leaves them open): the
  population standard deviation over the present fitted values, sums taken in
  row order; "rounded to p decimals" as rint(z * 10^p), half to even, kept as
  that integer; a column with zero deviation maps every value to token 0; a
  non-finite value, or a token the fitted rows never had, is missing.
* ``filter_contradictions``: the anti-contradiction stage of the Section 4
  preprocessing pipeline.  Reading: records with the same itemset and opposite
  labels contradict; mode 0 drops them in attack/normal pairs (k-th attack
  with k-th normal, record order), mode 1 drops every such record.
* ``evaluate``: the metrics of Section 4 / Table 2 (attack = positive); the
  AUC of the continuous score A - N (the paper does not name its score),
  counted pair by pair, ties one half.
* ``reg3_sweep``: labels of Regulations 1-3 for several r, then ``evaluate``.
"""
from __future__ import annotations

import bisect
import math

import numpy as np

MISSING = 0xFFFF


def _column_stats(column):
    """Population mean and deviation of the finite values, in row order."""
    total = 0.0
    count = 0
    for x in column:
        x = float(x)
        if math.isfinite(x):
            total = total + x
            count += 1
    if count == 0:
        return 0.0, 0.0
    mu = total / float(count)
    ss = 0.0
    for x in column:
        x = float(x)
        if math.isfinite(x):
            d = x - mu
            ss = ss + d * d
    return mu, math.sqrt(ss / float(count))


def _token(x, categorical, mu, sigma, scale):
    """Token of one value, or None when it is missing."""
    x = float(x)
    if not math.isfinite(x):
        return None
    if categorical:
        return x + 0.0                      # -0.0 and 0.0 are one value
    if not sigma > 0.0:
        return 0
    zs = ((x - mu) / sigma) * scale
    if not math.isfinite(zs) or abs(zs) >= 2.0 ** 62:
        raise OverflowError("z-score token out of range")
    return int(np.rint(zs))


def discretize(fit_values, categorical, p, values=None):
    """(codes uint16[n, F], cards uint16[F]) -- Section 3.1 tokens per column."""
    fit = np.asarray(fit_values, dtype=np.float64)
    vals = fit if values is None else np.asarray(values, dtype=np.float64)
    n_fit, F = fit.shape
    scale = float(10 ** int(p))
    codes = np.full(vals.shape, MISSING, dtype=np.uint16)
    cards = np.zeros(F, dtype=np.uint16)
    for f in range(F):
        cat = bool(categorical[f])
        mu, sigma = (0.0, 0.0) if cat else _column_stats(fit[:, f])
        vocab = set()
        for i in range(n_fit):
            t = _token(fit[i, f], cat, mu, sigma, scale)
            if t is not None:
                vocab.add(t)
        if len(vocab) > 65535:
            raise OverflowError("more than 65535 tokens in a column")
        rank = {t: k for k, t in enumerate(sorted(vocab))}
        cards[f] = len(vocab)
        for i in range(vals.shape[0]):
            try:
                t = _token(vals[i, f], cat, mu, sigma, scale)
            except OverflowError:
                t = None
            if t is not None and t in rank:
                codes[i, f] = rank[t]
    return codes, cards


def filter_contradictions(rows, labels, mode=0):
    """bool[n]: records kept after dropping contradicting ones."""
    rows = np.asarray(rows, dtype=np.uint64)
    labels = np.asarray(labels)
    by_itemset = {}
    for i in range(rows.shape[0]):
        key = tuple(int(w) for w in rows[i])
        by_itemset.setdefault(key, ([], []))[int(labels[i])].append(i)
    keep = np.ones(rows.shape[0], dtype=bool)
    for normal, attack in by_itemset.values():
        if mode == 0:
            k = min(len(normal), len(attack))
            dropped = normal[:k] + attack[:k]
        else:
            dropped = normal + attack if normal and attack else []
        for i in dropped:
            keep[i] = False
    return keep


def _ratio(a, b):
    return a / b if b else float("nan")


def auc_two_u(y_true, A, N):
    """(2U, n_attack, n_normal): 2U counts 2 per attack/normal pair with the
    attack record scoring higher on s = A - N, 1 per tie."""
    s = [int(a) - int(n) for a, n in zip(A, N)]
    pos = sorted(s[i] for i in range(len(s)) if y_true[i])
    neg = sorted(s[i] for i in range(len(s)) if not y_true[i])
    two_u = 0
    for v in pos:
        below = bisect.bisect_left(neg, v)
        upto = bisect.bisect_right(neg, v)
        two_u += 2 * below + (upto - below)
    return two_u, len(pos), len(neg)


def auc_brute(y_true, A, N):
    """The same count over every pair, for small inputs."""
    two_u = n_pos = n_neg = 0
    for i in range(len(y_true)):
        if not y_true[i]:
            continue
        for j in range(len(y_true)):
            if y_true[j]:
                continue
            si, sj = int(A[i]) - int(N[i]), int(A[j]) - int(N[j])
            two_u += 2 if si > sj else (1 if si == sj else 0)
    n_pos = int(sum(1 for y in y_true if y))
    n_neg = len(y_true) - n_pos
    return two_u, n_pos, n_neg


def evaluate(y_true, y_pred, A=None, N=None):
    yt = [int(v) for v in np.asarray(y_true)]
    yp = [int(v) for v in np.asarray(y_pred)]
    tp = sum(1 for t, p in zip(yt, yp) if t and p)
    fp = sum(1 for t, p in zip(yt, yp) if not t and p)
    tn = sum(1 for t, p in zip(yt, yp) if not t and not p)
    fn = sum(1 for t, p in zip(yt, yp) if t and not p)
    out = {"tp": tp, "fp": fp, "tn": tn, "fn": fn,
           "accuracy": _ratio(tp + tn, len(yt)),
           "precision": _ratio(tp, tp + fp),
           "recall": _ratio(tp, tp + fn),
           "f1": _ratio(2 * tp, 2 * tp + fp + fn),
           "auc": float("nan")}
    if A is not None and len(yt):
        two_u, n_pos, n_neg = auc_two_u(yt, np.asarray(A), np.asarray(N))
        if n_pos and n_neg:
            out["auc"] = float(two_u) / (2.0 * float(n_pos) * float(n_neg))
    return out


def reg3_sweep(A, N, y_true, mu, sigma, rs):
    """Regulations 1-3 for each r: attack if A >= N, A == N == 0, or
    N < mu - (r * sigma) in double precision."""
    out = []
    for r in rs:
        thr = mu - (float(r) * sigma)
        pred = [1 if (int(a) >= int(n) or (int(a) == 0 and int(n) == 0)
                      or float(int(n)) < thr) else 0
                for a, n in zip(A, N)]
        d = evaluate(y_true, pred, A, N)
        d["r"] = float(r)
        out.append(d)
    return out
