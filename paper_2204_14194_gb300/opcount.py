"""Operation counts of Table I (Sec. IV), used for algorithmic op accounting.

Counts are for one block with an M x N extrapolation area, a dictionary of
K = |D| atoms and I iterations; MUL, ADD and OTHER (divisions, comparisons,
square roots) are summed as the paper's Fig. 3 does.
"""
from __future__ import annotations


def se_ops(M: int, N: int, K: int, I: int) -> dict:
    """Original SE (Alg. 1), Table I top block."""
    MN = M * N
    return {"mul": I * (6 * MN * K + K + 2 * MN + 1),
            "add": I * (3 * MN * K + 2 * MN),
            "other": 3 * I * K}


def fase_ops(M: int, N: int, K: int, I: int) -> dict:
    """Fast SE (Alg. 3) without the tables, Table I middle block."""
    MN = M * N
    return {"mul": 2 * MN * K + I * (2 * K + MN + 1),
            "add": MN * K + I * (K + MN),
            "other": 2 * I * K}


def table_ops(M: int, N: int, K: int) -> dict:
    """Table generation (Alg. 2), Table I bottom block."""
    MN = M * N
    t = (K * K + K) * MN
    return {"mul": t, "add": t // 2, "other": t // 2 + K}


def total(d: dict) -> int:
    return int(d["mul"] + d["add"] + d["other"])


def fase_iteration_ops(M: int, N: int, K: int) -> int:
    """Per-iteration part of the FaSE count: 5K + 2MN + 1 operations."""
    return 5 * K + 2 * M * N + 1


def fase_iteration_ops_classes(M: int, N: int, K: int, classes: int = 4) -> int:
    """The same count when C(k,u) vanishes outside the selected atom's class
    (symmetric weighting, parity-structured atoms): the update, the scores and
    the maximum touch K / classes atoms per iteration, plus one comparison per
    class for the overall maximum."""
    return 5 * (K // classes) + classes + 2 * M * N + 1


def fase_select_update_ops(M: int, N: int, K: int, classes: int = 1) -> int:
    """The part of the per-iteration count that the iteration kernels execute:
    scores, maximum, coefficient and the update of eq. (20), without the 2MN
    operations of the model accumulate g += c phi_u (eq. 9), which the model
    kernel evaluates once from the selection log.  With parity classes the
    scores and the update touch K / classes atoms, plus one comparison per class."""
    if classes == 1:
        return fase_iteration_ops(M, N, K) - 2 * M * N
    return fase_iteration_ops_classes(M, N, K, classes) - 2 * M * N
