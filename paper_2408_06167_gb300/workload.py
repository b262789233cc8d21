"""Seeded synthetic biometric features (shared input generator; no HE arithmetic).

Stand-ins for the paper's face (IJB-C, LFW, ...) and fingerprint (PolyU,
FVC, ...) feature sets of Sec. 5.2, which are not available here: features are
i.i.d. N(0, 1) per dimension, then L2-normalised (ArcFace-style embeddings are
compared by cosine similarity, Sec. 2.2); each query is a gallery template
plus N(0, 0.3^2) noise per dimension, renormalised.  Seeds: gallery 1, query
choice and noise 2.
"""
from dataclasses import dataclass

import numpy as np

GALLERY_SEED = 1
QUERY_SEED = 2


def l2_normalise(x):
    x = np.asarray(x, dtype=np.float64)
    return x / np.linalg.norm(x, axis=-1, keepdims=True)


def gallery(n_ids, dim, seed=GALLERY_SEED):
    """(n_ids, dim) float64 L2-normalised Gaussian templates."""
    rng = np.random.default_rng(seed)
    return l2_normalise(rng.standard_normal((n_ids, dim)))


def queries(feats, n_queries, noise=0.3, seed=QUERY_SEED):
    """(n_queries, dim) probes: a uniformly chosen template + N(0, noise^2), renormalised.
    Returns (probes, true_ids)."""
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, len(feats), size=n_queries)
    q = feats[ids] + noise * rng.standard_normal((n_queries, feats.shape[1]))
    return l2_normalise(q), ids


def plaintext_scores(feats, q):
    """FP64 cosine similarity of unit vectors: <q, g_u> for every identity u."""
    return feats @ q


@dataclass(frozen=True)
class Workload:
    """One match workload: ring preset, feature dim, part size, gallery and batch size."""
    name: str
    preset: str
    dim: int
    part: int
    n_ids: int
    n_queries: int
    query_mode: str = "tiled"      # "tiled": one ct per query; "expanded": N_in cts per query


WORKLOADS = {
    "toy-16d-512": Workload("toy-16d-512", "toy", 16, 4, 512, 8, "expanded"),
    "face-128d-6144": Workload("face-128d-6144", "ring16", 128, 16, 6144, 1),
    "finger-16d-65536-q64": Workload("finger-16d-65536-q64", "ring16", 16, 4, 65536, 64),
    "large-128d-1m-q256": Workload("large-128d-1m-q256", "ring16", 128, 16, 1 << 20, 256),
    # one 65,536-row pack of the large workload with 32 queries: the same key-switch launch
    # shapes (128 ciphertexts a launch) on a device footprint small enough for counter captures
    "large-128d-64k-q32": Workload("large-128d-64k-q32", "ring16", 128, 16, 1 << 16, 32),
}
