"""Section 4 measurements made on a label array -- TEST INFRASTRUCTURE.

Plain numpy over labels produced by either side: cluster counts, cluster
sizes, the spanning test behind the R_span(p) curves (Section 4, Figs. 5-6)
and the size of the centre site's cluster on a Bethe lattice.
"""
from __future__ import annotations

import math

import numpy as np


def n_clusters(labels: np.ndarray) -> int:
    """Clusters are in one-to-one correspondence with sites that are their own label."""
    return int(np.count_nonzero(labels == np.arange(labels.size, dtype=labels.dtype)))


def cluster_sizes(labels: np.ndarray) -> np.ndarray:
    return np.bincount(labels, minlength=labels.size)


def sequential(labels: np.ndarray):
    """Clusters numbered 0..C-1 in the order of their smallest sites, and their
    sizes: np.unique sorts the distinct canonical labels ascending."""
    uniq, inverse, counts = np.unique(labels, return_inverse=True, return_counts=True)
    return inverse.astype(np.int32), counts.astype(np.int32)


def spanning_label(labels: np.ndarray, top: np.ndarray, bottom: np.ndarray) -> int:
    """The smallest label present among both the top and the bottom sites, or -1."""
    both = np.intersect1d(labels[top], labels[bottom])
    return int(both.min()) if both.size else -1


def spans(labels: np.ndarray, top: np.ndarray, bottom: np.ndarray) -> bool:
    """A cluster spans if it holds a site of the first row and one of the last
    row (open boundaries in the spanning direction, periodic across it)."""
    return bool(np.intersect1d(labels[top], labels[bottom]).size > 0)


def binomial_halfwidth(prob: float, samples: int, sigmas: float = 4.0) -> float:
    return sigmas * math.sqrt(max(prob * (1 - prob), 1e-12) / samples)
