"""Seeded synthetic IG workloads shaped like the paper's intrusion-detection data.

This module only draws inputs: per-feature integer codes (already discretised
bins), class labels and train/test splits.  It holds none of the method's
arithmetic -- no encoding to bitsets, no intersections, no subset tests, no
scores -- so both the CPU oracle and the CUDA path can take their inputs from
it without sharing any computation.

The paper evaluates on NSL-KDD (41 features, Section 4), UNSW-NB15 and
UKM-IDS20; none of those datasets is available here, so these seeded
generators stand in for them, reproducing only shapes, sizes and the kind of
skew (many zero-dominated numeric columns, a few high-cardinality categorical
ones, class-conditional value distributions that partly overlap).

Every random draw goes through ``numpy.random.Generator(PCG64(seed))`` with the
seed fixed per workload, so a workload is a pure function of its name.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

NORMAL = 0
ATTACK = 1

# NSL-KDD-like feature cardinalities: protocol_type (3), service (70),
# flag (11), then 38 numeric columns quantile-binned to 10 bins each.
NSL_CARDS = [3, 70, 11] + [10] * 38


@dataclass
class Workload:
    """One IG problem: codes[i, f] is the bin of feature f in record i."""

    name: str
    cards: np.ndarray            # uint16[F]
    train_codes: np.ndarray      # uint16[n_train, F]
    train_labels: np.ndarray     # uint8[n_train], 1 = attack, 0 = normal
    test_codes: np.ndarray       # uint16[n_test, F]
    test_labels: np.ndarray      # uint8[n_test]
    meta: dict = field(default_factory=dict)

    @property
    def n_features(self) -> int:
        return int(self.cards.shape[0])

    @property
    def n_items(self) -> int:
        """L, the size of the item universe: one item per (feature, bin)."""
        return int(self.cards.astype(np.int64).sum())

    @property
    def n_words(self) -> int:
        """K = ceil(L / 64) packed 64-bit words per record."""
        return (self.n_items + 63) // 64


def zipf_pmf(card: int, s: float) -> np.ndarray:
    """Zipf(s) probabilities over ranks 1..card (largest mass first)."""
    ranks = np.arange(1, card + 1, dtype=np.float64)
    p = ranks ** (-float(s))
    return p / p.sum()


def class_pmfs(rng: np.random.Generator, cards, exponents, shared_frac: float):
    """Per-class categorical distributions for every feature.

    For feature f a shared Zipf pmf (placed on the bins by one seeded
    permutation) is mixed with a class-specific Zipf pmf (placed by an
    independent permutation per class): p_c = shared*Z_shared + (1-shared)*Z_c.
    Returns {NORMAL: [pmf_f ...], ATTACK: [pmf_f ...]}.
    """
    out = {NORMAL: [], ATTACK: []}
    for card, s in zip(cards, exponents):
        base = zipf_pmf(int(card), s)
        shared = base[rng.permutation(int(card))]
        for c in (NORMAL, ATTACK):
            own = base[rng.permutation(int(card))]
            p = shared_frac * shared + (1.0 - shared_frac) * own
            out[c].append(p / p.sum())
    return out


def draw_codes(rng: np.random.Generator, pmfs, n: int) -> np.ndarray:
    """n records, each feature drawn independently from its class pmf."""
    F = len(pmfs)
    codes = np.empty((n, F), dtype=np.uint16)
    for f, p in enumerate(pmfs):
        codes[:, f] = rng.choice(p.shape[0], size=n, p=p).astype(np.uint16)
    return codes


def _mixed(rng, pmfs, n_normal: int, n_attack: int):
    """Draw both classes and interleave them by a seeded permutation."""
    codes = np.concatenate([draw_codes(rng, pmfs[NORMAL], n_normal),
                            draw_codes(rng, pmfs[ATTACK], n_attack)])
    labels = np.concatenate([np.full(n_normal, NORMAL, np.uint8),
                             np.full(n_attack, ATTACK, np.uint8)])
    order = rng.permutation(codes.shape[0])
    return np.ascontiguousarray(codes[order]), np.ascontiguousarray(labels[order])


def tiny(seed: int = 1001) -> Workload:
    """500 train (250/250) + 2,000 test records; 16 features x 16 bins.

    Zipf(s=1.2) bins per class with 30% shared mass: L = 256 items, K = 4.
    The test set is 53% normal.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cards = [16] * 16
    pmfs = class_pmfs(rng, cards, [1.2] * 16, shared_frac=0.3)
    tr_c, tr_l = _mixed(rng, pmfs, 250, 250)
    te_c, te_l = _mixed(rng, pmfs, 1060, 940)
    return Workload("ig-tiny-500x16x16", np.asarray(cards, np.uint16),
                    tr_c, tr_l, te_c, te_l,
                    {"seed": seed, "zipf_s": 1.2, "shared_frac": 0.3})


# Calibration of the NSL-KDD-shaped generator (fixed once, then frozen).
#
# Records are drawn from a latent mixture of NSL_PROTOTYPES prototype flows,
# shared between the classes (class weights = NSL_PROTO_SHARED of a common
# Zipf(NSL_PROTO_S) weighting + the rest a class-specific one).  A record
# copies its prototype's bin on feature f with probability rho_f ~
# U[NSL_RHO_LO, NSL_RHO_HI] and otherwise draws the bin from its class pmf
# (Zipf with exponent U[NSL_S_LO, NSL_S_HI] per feature, NSL_SHARED_FRAC
# of it class-independent).  With independent features alone, almost every
# pairwise intersection is unique and coherent (about 1.3e7 coherent patterns
# at 15k records, 60x the paper's NSL-KDD 5|5 count of 210,448 in Table 1);
# the prototype layer reproduces the redundancy of real flow records and puts
# the 15k workload at a few 1e5 coherent patterns.
NSL_S_LO = 1.0
NSL_S_HI = 2.5
NSL_SHARED_FRAC = 0.5
NSL_PROTOTYPES = 64
NSL_PROTO_S = 1.1
NSL_PROTO_SHARED = 0.8
NSL_RHO_LO = 0.9
NSL_RHO_HI = 1.0


def _prototype_records(rng, protos, weights, rho, pmfs, n):
    """n records: prototype bins, each resampled from pmfs with prob 1-rho_f."""
    z = rng.choice(protos.shape[0], size=n, p=weights)
    codes = protos[z].copy()
    noise = draw_codes(rng, pmfs, n)
    resample = rng.random((n, protos.shape[1])) >= rho[None, :]
    codes[resample] = noise[resample]
    return codes


class _NslSampler:
    """Draws NSL-KDD-shaped records of either class (see nsl_like)."""

    def __init__(self, rng: np.random.Generator):
        self.rng = rng
        self.cards = NSL_CARDS
        F = len(self.cards)
        exps = rng.uniform(NSL_S_LO, NSL_S_HI, size=F)
        self.pmfs = class_pmfs(rng, self.cards, exps, shared_frac=NSL_SHARED_FRAC)
        mean_pmfs = [0.5 * (self.pmfs[NORMAL][f] + self.pmfs[ATTACK][f]) for f in range(F)]
        mean_pmfs = [p / p.sum() for p in mean_pmfs]
        self.protos = draw_codes(rng, mean_pmfs, NSL_PROTOTYPES)
        base = zipf_pmf(NSL_PROTOTYPES, NSL_PROTO_S)
        common = base[rng.permutation(NSL_PROTOTYPES)]
        self.weights = {}
        for c in (NORMAL, ATTACK):
            w = NSL_PROTO_SHARED * common + (1.0 - NSL_PROTO_SHARED) * base[
                rng.permutation(NSL_PROTOTYPES)]
            self.weights[c] = w / w.sum()
        self.rho = rng.uniform(NSL_RHO_LO, NSL_RHO_HI, size=F)

    def draw(self, c: int, n: int) -> np.ndarray:
        return _prototype_records(self.rng, self.protos, self.weights[c], self.rho,
                                  self.pmfs[c], n)


def nsl_like(n_records: int, train_frac: float, seed: int, name: str,
             normal_frac: float = 0.53) -> Workload:
    """NSL-KDD-shaped records: 41 features, 464 items, K = 8 words.

    Class counts are stratified exactly: round(normal_frac * n) normal records
    overall, and the same fraction (rounded) within the training split.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sampler = _NslSampler(rng)
    cards = NSL_CARDS

    n_train = int(round(train_frac * n_records))
    n_normal = int(round(normal_frac * n_records))
    tr_normal = int(round(normal_frac * n_train))
    tr_attack = n_train - tr_normal
    te_normal = n_normal - tr_normal
    te_attack = (n_records - n_train) - te_normal

    def split(n_norm, n_att):
        codes = np.concatenate([sampler.draw(NORMAL, n_norm), sampler.draw(ATTACK, n_att)])
        labels = np.concatenate([np.full(n_norm, NORMAL, np.uint8),
                                 np.full(n_att, ATTACK, np.uint8)])
        order = rng.permutation(codes.shape[0])
        return (np.ascontiguousarray(codes[order]),
                np.ascontiguousarray(labels[order]))

    tr_c, tr_l = split(tr_normal, tr_attack)
    te_c, te_l = split(te_normal, te_attack)
    return Workload(name, np.asarray(cards, np.uint16), tr_c, tr_l, te_c, te_l,
                    {"seed": seed, "zipf_s_range": [NSL_S_LO, NSL_S_HI],
                     "shared_frac": NSL_SHARED_FRAC,
                     "prototypes": NSL_PROTOTYPES, "proto_s": NSL_PROTO_S,
                     "proto_shared": NSL_PROTO_SHARED,
                     "rho_range": [NSL_RHO_LO, NSL_RHO_HI],
                     "normal_frac": normal_frac, "train_frac": train_frac})


def nsl15k(seed: int = 1002) -> Workload:
    """15,000 records (53% normal), 50/50 train/test split."""
    return nsl_like(15000, 0.5, seed, "ig-nsl-15k-50/50")


def nsl148k(seed: int = 1003) -> Workload:
    """148,000 records (53% normal), 10% train / 90% test."""
    return nsl_like(148000, 0.1, seed, "ig-nsl-148k-10/90")


def batched_problem(i: int, base_seed: int = 2000) -> Workload:
    """Problem i of the batched workload (64 problems).

    Record count log-uniform in [200, 8000], itemset width in
    {128, 256, 512, 1024} bits (width/16 features of 16 bins, Zipf(1.2),
    30% shared), attack fraction uniform in [0.3, 0.7]; 10% of the records
    are held out as test.
    """
    rng = np.random.Generator(np.random.PCG64(base_seed + i))
    n = int(round(np.exp(rng.uniform(np.log(200.0), np.log(8000.0)))))
    width = int(rng.choice([128, 256, 512, 1024]))
    attack_frac = float(rng.uniform(0.3, 0.7))
    F = width // 16
    cards = [16] * F
    pmfs = class_pmfs(rng, cards, [1.2] * F, shared_frac=0.3)
    n_test = n // 10
    n_train = n - n_test
    tr_attack = int(round(attack_frac * n_train))
    te_attack = int(round(attack_frac * n_test))
    tr_c, tr_l = _mixed(rng, pmfs, n_train - tr_attack, tr_attack)
    te_c, te_l = _mixed(rng, pmfs, n_test - te_attack, te_attack)
    return Workload(f"ig-batched-{i}", np.asarray(cards, np.uint16),
                    tr_c, tr_l, te_c, te_l,
                    {"seed": base_seed + i, "width": width,
                     "attack_frac": attack_frac})


def random_words(rng: np.random.Generator, n: int, n_items: int,
                 density: str = "half") -> np.ndarray:
    """Arbitrary (not one-hot) itemsets as uint64[n, ceil(n_items/64)].

    Uniform random words, thinned ("quarter": AND of two draws, "eighth":
    AND of three) or thickened ("three_quarters": OR of two draws); every bit
    at a position >= n_items is cleared.  Used for small adversarial cases that the one-hot
    generators cannot produce.
    """
    K = (n_items + 63) // 64
    hi = np.iinfo(np.uint64).max

    def draw():
        return rng.integers(0, hi, size=(n, K), dtype=np.uint64, endpoint=True)

    w = draw()
    if density == "quarter":
        w &= draw()
    elif density == "eighth":
        w &= draw()
        w &= draw()
    elif density == "three_quarters":
        w |= draw()
    elif density != "half":
        raise ValueError(density)
    for k in range(K):
        lo = 64 * k
        if n_items <= lo:
            w[:, k] = 0
        elif n_items < lo + 64:
            w[:, k] &= np.uint64((1 << (n_items - lo)) - 1)
    return w


WORKLOADS = {
    "tiny": tiny,
    "nsl15k": nsl15k,
    "nsl148k": nsl148k,
}

BATCHED_PROBLEMS = 64


def batched(count: int = BATCHED_PROBLEMS, base_seed: int = 2000) -> list:
    """The batched workload: `count` independent problems (batched_problem)."""
    return [batched_problem(i, base_seed) for i in range(count)]


MISSING = 0xFFFF  # code of a missing value: the feature contributes no item


@dataclass
class ServedWorkload:
    """Pattern sets to serve, flows to score and a request stream."""

    name: str
    cards: np.ndarray
    patterns: dict         # class -> uint16[P, F] codes, MISSING where dropped
    support: dict          # class -> uint32[P]
    flow_codes: np.ndarray  # uint16[total_flows, F]
    request_sizes: np.ndarray  # int64[R], summing to total_flows
    unit_gaps: np.ndarray   # float64[R], Exp(1) inter-arrival gaps (unit rate)
    meta: dict = field(default_factory=dict)


def _unique_rows(a: np.ndarray) -> np.ndarray:
    """np.unique(a, axis=0) for a uint16 matrix -- the distinct rows in
    ascending lexicographic order -- computed on one byte string per row
    (big-endian, so that byte order is numeric order), which sorts much
    faster than the column-wise row comparison."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    keys = np.ascontiguousarray(a.astype(">u2")).view(np.dtype((np.void, 2 * a.shape[1])))
    return np.unique(keys.ravel()).view(">u2").reshape(-1, a.shape[1]).astype(np.uint16)


def served(per_class: int = 1_000_000, total_flows: int = 1_000_000, seed: int = 1005,
           keep_frac: float = 0.5, max_request: int = 4096) -> ServedWorkload:
    """The served-scoring workload (NSL-KDD-shaped, K = 8).

    Each pattern is a record of its class drawn from the NSL-KDD-shaped
    generator with every feature kept with probability keep_frac and the
    others marked MISSING (at least one kept); patterns are distinct as code
    rows, per_class of them per class.  Supports are uniform in 1..1000.
    Flows are records of both classes (53% normal).  Requests carry
    log-uniform sizes in [1, max_request] flows until total_flows are used;
    their arrival gaps are unit-rate exponentials (a Poisson stream, scaled
    to the wanted rate by the caller).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sampler = _NslSampler(rng)
    patterns, support = {}, {}
    for c in (NORMAL, ATTACK):
        have = np.empty((0, len(NSL_CARDS)), np.uint16)
        while have.shape[0] < per_class:
            need = int((per_class - have.shape[0]) * 1.3) + 1024
            codes = sampler.draw(c, need)
            keep = rng.random(codes.shape) < keep_frac
            keep[np.arange(need), rng.integers(0, codes.shape[1], need)] = True
            codes = np.where(keep, codes, np.uint16(MISSING)).astype(np.uint16)
            have = _unique_rows(np.concatenate([have, codes]))
        patterns[c] = np.ascontiguousarray(have[rng.permutation(have.shape[0])[:per_class]])
        support[c] = rng.integers(1, 1001, size=per_class).astype(np.uint32)
    n_normal = int(round(0.53 * total_flows))
    flows = np.concatenate([sampler.draw(NORMAL, n_normal),
                            sampler.draw(ATTACK, total_flows - n_normal)])
    flows = np.ascontiguousarray(flows[rng.permutation(total_flows)])
    sizes = []
    left = total_flows
    while left > 0:
        m = int(round(np.exp(rng.uniform(0.0, np.log(max_request)))))
        m = max(1, min(m, left))
        sizes.append(m)
        left -= m
    sizes = np.asarray(sizes, np.int64)
    gaps = rng.exponential(1.0, size=sizes.shape[0])
    return ServedWorkload(f"ig-served-{per_class}x2-patterns-{total_flows}-flows",
                          np.asarray(NSL_CARDS, np.uint16), patterns, support, flows,
                          sizes, gaps, {"seed": seed, "keep_frac": keep_frac,
                                        "max_request": max_request})


@dataclass
class RawFlows:
    """Raw (undiscretised) flow attributes for the preprocessing helpers."""

    values: np.ndarray       # float64[n, F]; NaN = missing
    categorical: np.ndarray  # bool[F]
    labels: np.ndarray       # uint8[n], 1 = attack


def raw_flows(n: int, seed: int = 1006, missing_frac: float = 0.001) -> RawFlows:
    """NSL-KDD-shaped raw attributes: 41 columns -- three categorical (3, 70
    and 11 values, as integer-valued floats), then 38 numeric ones of three
    kinds drawn per class: zero-inflated log-normal byte/duration counts,
    rates in [0, 1] with two decimals, and small Poisson counts.  A fraction
    `missing_frac` of all entries is NaN.  Labels are 53% normal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    labels = (rng.random(n) >= 0.53).astype(np.uint8)
    F = 41
    vals = np.empty((n, F), np.float64)
    cat = np.zeros(F, bool)
    cat[:3] = True
    for f, card in enumerate((3, 70, 11)):
        pmf = [rng.dirichlet(np.full(card, 0.3)) for _ in range(2)]
        for c in (0, 1):
            idx = np.flatnonzero(labels == c)
            vals[idx, f] = rng.choice(card, size=idx.size, p=pmf[c]).astype(np.float64)
    for f in range(3, F):
        kind = f % 3
        for c in (0, 1):
            idx = np.flatnonzero(labels == c)
            m = idx.size
            if kind == 0:
                zero = rng.random() * 0.9
                mean, sd = rng.uniform(2.0, 8.0), rng.uniform(0.5, 2.0)
                v = np.round(rng.lognormal(mean, sd, m))
                v[rng.random(m) < zero] = 0.0
            elif kind == 1:
                a, b = rng.uniform(0.2, 3.0, 2)
                v = np.round(rng.beta(a, b, m), 2)
            else:
                v = rng.poisson(rng.uniform(0.1, 20.0), m).astype(np.float64)
            vals[idx, f] = v
    vals[rng.random((n, F)) < missing_frac] = np.nan
    return RawFlows(vals, cat, labels)
