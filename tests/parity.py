"""Helpers that run the FP64 oracle and the CUDA library side by side on the same seeded slices.

Not a test module: imported by the GPU parity tests.
"""

from __future__ import annotations

import math

import numpy as np

import oracle as O


def decision_margins(log: dict, tau_rel_rank: bool = True) -> float:
    """Smallest relative distance |stat - eps^2| / eps^2 of the update's decisions: the
    ||E_k|| <= eps tests, the rank cuts (tail sums at the chosen rank and one below) and q <= eps."""
    eps2 = log["eps"] ** 2
    if eps2 == 0.0:
        return math.inf
    ms = []
    for m in log["modes"]:
        ms.append(abs(m.e_norm2 - eps2) / eps2)
        if m.grew and m.lam is not None:
            lam = m.lam
            tails = np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])
            ms.append(abs(tails[m.r_add] - eps2) / eps2)
            if m.r_add >= 1:
                ms.append(abs(tails[m.r_add - 1] - eps2) / eps2)
    ms.append(abs(log["isvd"].q ** 2 - eps2) / eps2)
    return min(ms)


def subspace_sin(Ua: np.ndarray, Ub: np.ndarray) -> float:
    """Largest principal-angle sine between the column spans (equal column counts)."""
    Qa, _ = np.linalg.qr(Ua)
    Qb, _ = np.linalg.qr(Ub)
    M = Qb - Qa @ (Qa.T @ Qb)
    return float(np.linalg.norm(M, 2)) if M.size else 0.0


def aligned_core_diff(C_o, Us_o, C_g, Us_g) -> float:
    """||C_o - C_g'|| / ||C_o|| after flipping the signs of C_g's mode-k slices so that
    diag(U_k,o^T U_k,g) > 0 (eigenvector sign freedom)."""
    Cg = C_g.copy()
    for k, (Uo, Ug) in enumerate(zip(Us_o, Us_g)):
        s = np.sign(np.sum(Uo * Ug, axis=0))
        s[s == 0] = 1.0
        Cg = O.ttm(Cg, np.diag(s), k)
    return float(np.linalg.norm(C_o - Cg) / np.linalg.norm(C_o))


def to_device(x: np.ndarray, dtype):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x.T)).to(dtype=dtype, device="cuda").contiguous()


def gpu_state_numpy(ts):
    import paper_2308_16395_gb300 as pkg  # noqa: F401

    C = ts.core().cpu().numpy()
    Us = [ts.factor(k).cpu().numpy() for k in range(ts.d)]
    return C, Us


def oracle_tails(m) -> np.ndarray:
    """Alg. 1's tails lambda_{l+1} + ... + lambda_n (l = 0..n) of a grown mode's residual Gram."""
    lam = np.asarray(m.lam)
    return np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])


def replay_for(log: dict, delta: float, delta_q: float | None = None):
    """The oracle's decisions of one update whose statistic lies within `delta` (relative) of
    eps^2 (`delta_q` for Alg. 3's q^2, default `delta`), as (grow, augment) arguments of
    tucker_replay_next; None when no decision is near.

    grow[k] is -1 (the library decides), 0 (no growth) or the oracle's r'_k; augment is -1 or the
    oracle's branch of Alg. 3 (reading of the paper on near-cutoff decisions under mixed
    precision: such a decision may come out either way, and the library is then made to take the
    oracle's so that the two stay comparable)."""
    eps2 = log["eps"] ** 2
    if eps2 == 0.0:
        return None
    near = False
    grow = []
    for m in log["modes"]:
        g = -1
        if abs(m.e_norm2 - eps2) / eps2 < delta:
            g = m.r_add if m.grew else 0
        elif m.grew and m.lam is not None:
            t = oracle_tails(m)
            if min(abs(t[m.r_add] - eps2), abs(t[m.r_add - 1] - eps2)) / eps2 < delta:
                g = m.r_add
        near |= g >= 0
        grow.append(g)
    aug = -1
    if abs(log["isvd"].q ** 2 - eps2) / eps2 < (delta if delta_q is None else delta_q):
        aug = int(log["isvd"].augmented)
        near = True
    return (grow, aug) if near else None
