"""Field-comparison metrics of Schrijver et al. (2006), used by the paper's Table 1 (Sect. 2.3).

B is the reconstructed field and b the reference field, both (M, 3):
  C_vec = sum B.b / sqrt(sum |B|^2 sum |b|^2)
  C_CS  = (1/M) sum B.b / (|B| |b|)
  E'_n  = 1 - sum |B - b| / sum |b|
  E'_m  = 1 - (1/M) sum |B - b| / |b|
  eps   = sum |B|^2 / sum |b|^2
Test infrastructure only (FP64 numpy)."""
from __future__ import annotations

import numpy as np


def field_metrics(B, b) -> dict:
    B = np.asarray(B, np.float64).reshape(-1, 3)
    b = np.asarray(b, np.float64).reshape(-1, 3)
    nB = np.linalg.norm(B, axis=1)
    nb = np.linalg.norm(b, axis=1)
    dot = np.sum(B * b, axis=1)
    err = np.linalg.norm(B - b, axis=1)
    return dict(
        C_vec=float(dot.sum() / np.sqrt((nB ** 2).sum() * (nb ** 2).sum())),
        C_cs=float(np.mean(dot / (nB * nb))),
        E_n=float(1.0 - err.sum() / nb.sum()),
        E_m=float(1.0 - np.mean(err / nb)),
        eps=float((nB ** 2).sum() / (nb ** 2).sum()),
    )
