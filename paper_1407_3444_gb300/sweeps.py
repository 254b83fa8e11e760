"""Comparison drivers of Sec. III over the library's static entry points (the band-pair
histogram of Fig. 8, the band-truncation and matrix-element studies).

- ``band_truncation``: static chi0(q) with the band sum restricted to windows around E_F
  (the convergence of chi0 with the number of bands, Sec. III; the paper's FeSe result needs
  about 50 bands);
- ``cma_vs_exact``: static chi0(q) with |M|^2 = 1 (the constant matrix element
  approximation) beside the exact |M|^2, the CMA curve also shifted to 0 at the first q, as
  the paper compares them (its background shift has no physical meaning);
- ``pair_contributions``: the band-pair histogram of chi0 at one q (Fig. 8).

Each runs whole calls of the C-ABI (``chi0.Plan``); nothing here computes chi0 itself."""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import chi0


def _static(W, qs, precision: str, window=None, cma=None, **kw) -> np.ndarray:
    P = chi0.Plan(W, precision=precision, device=True, window=window, cma=cma, qs=qs, **kw)
    try:
        out = P.static()
        return out.cpu().numpy() if hasattr(out, "cpu") else np.asarray(out)
    finally:
        P.close()


def band_truncation(W, qs: Sequence, widths: Sequence[int], precision: str = "mixed") -> Dict[int, np.ndarray]:
    """chi0(q) for band windows of the given widths centred on the Fermi level (the bands of
    the window around the highest occupied band, clamped to the workload's bands)."""
    nocc = int(np.round(np.mean(np.sum(W.E < W.ef, axis=1))))
    out = {}
    for w in widths:
        w = int(min(max(w, 1), W.nb))
        lo = int(min(max(nocc - w // 2, 0), W.nb - w))
        out[w] = _static(W, qs, precision, window=(lo, lo + w))
    return out


def cma_vs_exact(W, qs: Sequence, window=None, precision: str = "mixed") -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(exact chi0(q), CMA chi0(q), CMA chi0(q) - CMA chi0(q_0))."""
    exact = _static(W, qs, precision, window=window, cma=False)
    cma = _static(W, qs, precision, window=window, cma=True)
    return exact, cma, cma - cma[0]


def pair_contributions(W, q, precision: str = "mixed", window=None) -> Tuple[float, np.ndarray]:
    """(chi0(q), [w, w] band-pair contributions, entry (m - lo, n - lo) for m -> n)."""
    P = chi0.Plan(W, precision=precision, device=True, window=window, qs=[q])
    try:
        chi, blocks = P.static_pairs()
        return float(chi[0]), blocks[0]
    finally:
        P.close()
