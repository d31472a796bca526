"""Section 4 measurements made on a label array -- TEST INFRASTRUCTURE.

Plain numpy over labels produced by either side: cluster counts, the
sequential numbering of clusters with their sizes (the renumbering at the end
of Section 3), the largest cluster, and the spanning test behind the
R_span(p) curves (Section 4, Figs. 5-6).
"""
from __future__ import annotations

import numpy as np


def n_clusters(labels: np.ndarray) -> int:
    """Clusters are in one-to-one correspondence with sites that are their own label."""
    return int(np.count_nonzero(labels == np.arange(labels.size, dtype=labels.dtype)))


def sequential(labels: np.ndarray):
    """Clusters numbered 0..C-1 in the order of their smallest sites, and their
    sizes: np.unique sorts the distinct canonical labels ascending."""
    uniq, inverse, counts = np.unique(labels, return_inverse=True, return_counts=True)
    return inverse.astype(np.int32), counts.astype(np.int32)


def largest_cluster(labels: np.ndarray) -> tuple[int, int]:
    """(size, label) of the largest cluster: the most frequent canonical label,
    the smallest such label on ties (np.argmax returns the first maximum);
    (0, -1) for no sites."""
    if labels.size == 0:
        return 0, -1
    counts = np.bincount(labels, minlength=labels.size)
    lab = int(np.argmax(counts))
    return int(counts[lab]), lab


def spanning_label(labels: np.ndarray, top: np.ndarray, bottom: np.ndarray) -> int:
    """The smallest label present among both the top and the bottom sites, or -1."""
    both = np.intersect1d(labels[top], labels[bottom])
    return int(both.min()) if both.size else -1


def spans(labels: np.ndarray, top: np.ndarray, bottom: np.ndarray) -> bool:
    """A cluster spans if it holds a site of the first row and one of the last
    row (open boundaries in the spanning direction, periodic across it)."""
    return bool(np.intersect1d(labels[top], labels[bottom]).size > 0)
