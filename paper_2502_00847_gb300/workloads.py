"""Seeded synthetic inputs (logit vectors) standing in for the paper's
workloads: no homomorphic arithmetic here, only random draws.

SecPE's experiments aggregate the logits of K prompted model runs over C
classes (GLUE tasks: C = 2..3 with 4 templates; self-consistency and CLIP:
many classes and 80..247 prompts).  Those datasets and model weights are not
available, so the logits are drawn from fixed distributions:

* toy:     K = 5 vectors of C = 2 classes, uniform in [-1, 1], redrawn until
           the top-2 gap of the mean vector is >= 0.05; public bounds [-1, 1].
* argmax:  per query K ~ U{4, 8, 16}, C ~ U{2, 3, 4, 6, 14, 64}; per-prompt
           logits N(0, 1) (float32) clipped to [-4, 4]; if the mean vector's
           top-1 gap is < 0.02, the gap is added to the top class of every
           prompt; public bounds [-4.25, 4.25].
* packed:  sets of inputs sharing a task (K, C drawn as above), as many per
           set as slot packing fits (or a fraction), each input drawn as an
           argmax query.
"""
from dataclasses import dataclass

import numpy as np

TOY_BOUNDS = (-1.0, 1.0)
ARGMAX_BOUNDS = (-4.25, 4.25)
ARGMAX_K = (4, 8, 16)
ARGMAX_C = (2, 3, 4, 6, 14, 64)


@dataclass
class Query:
    logits: np.ndarray  # [K][C] float64
    d_min: float
    d_max: float
    qseed: int
    enc_seeds: list     # one encryption seed per prompt

    @property
    def K(self):
        return self.logits.shape[0]

    @property
    def C(self):
        return self.logits.shape[1]


def toy_query(seed=1, K=5, C=2):
    rng = np.random.default_rng(seed)
    while True:
        logits = rng.uniform(-1.0, 1.0, (K, C))
        srt = np.sort(logits.mean(0))
        if srt[-1] - srt[-2] >= 0.05:
            break
    return Query(logits, TOY_BOUNDS[0], TOY_BOUNDS[1], qseed=seed * 7919 + 1,
                 enc_seeds=[seed * 1000 + i for i in range(K)])


def argmax_queries(n_queries, seed=4, K_choices=ARGMAX_K, C_choices=ARGMAX_C, margin=0.02):
    rng = np.random.default_rng(seed)
    out = []
    for qi in range(n_queries):
        K = int(rng.choice(K_choices))
        C = int(rng.choice(C_choices))
        logits = np.clip(rng.standard_normal((K, C)).astype(np.float32), -4.0, 4.0).astype(np.float64)
        mean = logits.mean(0)
        top = int(np.argmax(mean))
        srt = np.sort(mean)
        gap = srt[-1] - srt[-2]
        if gap < margin:
            logits[:, top] += margin - gap
        out.append(Query(logits, ARGMAX_BOUNDS[0], ARGMAX_BOUNDS[1], qseed=(seed << 32) + qi,
                         enc_seeds=[(seed << 40) + (qi << 8) + i for i in range(K)]))
    return out


@dataclass
class PackedQuery:
    """P inputs of one task (same C and prompt ensemble K) that share one
    ciphertext per prompt under slot packing."""
    logits: np.ndarray  # [P][K][C] float64
    d_min: float
    d_max: float
    qseed: int
    enc_seeds: list     # one encryption seed per prompt (ciphertext)

    @property
    def P(self):
        return self.logits.shape[0]

    @property
    def K(self):
        return self.logits.shape[1]

    @property
    def C(self):
        return self.logits.shape[2]

    def prompt(self, i):
        """[P][C]: prompt i's logits of every input (ciphertext i's content)."""
        return np.ascontiguousarray(self.logits[:, i, :])


def packed_queries(n_sets, slots, seed=6, K_choices=ARGMAX_K, C_choices=ARGMAX_C, margin=0.02, fill=1.0):
    """Packed query sets with the Argmax mix's task distribution: each set
    draws K and C like one query of the mix and holds round(fill * slots /
    (2 C')) inputs, each input drawn like a query of the mix (N(0,1) float32
    logits clipped to [-4, 4], top-1 mean gap planted to >= margin)."""
    rng = np.random.default_rng(seed)
    out = []
    for si in range(n_sets):
        K = int(rng.choice(K_choices))
        C = int(rng.choice(C_choices))
        cp = 1 << (C - 1).bit_length()
        P = max(1, int(round(fill * (slots // (2 * cp)))))
        logits = np.clip(rng.standard_normal((P, K, C)).astype(np.float32), -4.0, 4.0).astype(np.float64)
        for b in range(P):
            mean = logits[b].mean(0)
            top = int(np.argmax(mean))
            srt = np.sort(mean)
            gap = srt[-1] - srt[-2]
            if gap < margin:
                logits[b, :, top] += margin - gap
        out.append(PackedQuery(logits, ARGMAX_BOUNDS[0], ARGMAX_BOUNDS[1], qseed=(seed << 32) + si,
                               enc_seeds=[(seed << 40) + (si << 8) + i for i in range(K)]))
    return out


@dataclass
class ClipTask:
    """CLIP-style zero-shot classification inputs (Sec. 2.3): an image
    embedding x[d] and plaintext text embeddings T[K][C][d] of K prompt
    templates and C classes, drawn so that the ensembled logits
    mean_i T_i x have a top-1 gap >= margin."""
    T: np.ndarray
    x: np.ndarray
    d_min: float
    d_max: float
    qseed: int
    enc_seed: int

    @property
    def K(self):
        return self.T.shape[0]

    @property
    def C(self):
        return self.T.shape[1]

    @property
    def d(self):
        return self.T.shape[2]

    def logits(self):
        return np.einsum("kcd,d->kc", self.T, self.x)


def clip_task(d=64, C=10, K=3, seed=7, margin=0.05):
    """Unit-norm embeddings (as CLIP normalises them) scaled so the logits
    stay well inside [-4.25, 4.25]; redrawn until the margin holds."""
    rng = np.random.default_rng(seed)
    while True:
        x = rng.standard_normal(d)
        x /= np.linalg.norm(x)
        base = rng.standard_normal((C, d))
        T = base[None] + 0.3 * rng.standard_normal((K, C, d))
        T /= np.linalg.norm(T, axis=2, keepdims=True)
        T *= 3.0
        mean = np.einsum("kcd,d->kc", T, x).mean(0)
        srt = np.sort(mean)
        if srt[-1] - srt[-2] >= margin:
            return ClipTask(T, x, ARGMAX_BOUNDS[0], ARGMAX_BOUNDS[1], qseed=seed * 7919 + 3, enc_seed=seed * 1000 + 1)


def clip_images(d=512, C=10, K=80, B=16, seed=8, margin=0.05):
    """One zero-shot task (text embeddings T[K][C][d] of K templates, as in
    CLIP's 80) and B image embeddings, each redrawn until its ensembled
    logits have a top-1 gap >= margin: returns (T, [x_b], qseeds, enc_seeds)."""
    rng = np.random.default_rng(seed)
    base = rng.standard_normal((C, d))
    T = base[None] + 0.3 * rng.standard_normal((K, C, d))
    T /= np.linalg.norm(T, axis=2, keepdims=True)
    T *= 3.0
    xs = []
    while len(xs) < B:
        x = rng.standard_normal(d)
        x /= np.linalg.norm(x)
        mean = np.einsum("kcd,d->kc", T, x).mean(0)
        srt = np.sort(mean)
        if srt[-1] - srt[-2] >= margin:
            xs.append(x)
    return T, xs, [(seed << 32) + b for b in range(B)], [(seed << 40) + b for b in range(B)]


def residues(shape, primes, seed):
    """Uniform residues [..., len(primes), N] for primitive micro-benchmarks."""
    rng = np.random.default_rng(seed)
    out = np.empty(shape, dtype=np.uint64)
    for i, q in enumerate(primes):
        out[..., i, :] = rng.integers(0, q, size=out[..., i, :].shape, dtype=np.uint64)
    return out
