"""Oracle: baseline-types and the two reduced redundant-calibration selections.

TEST INFRASTRUCTURE ONLY: the library's product path never imports this
module, and this module imports nothing from the library.

Paper basis:
  * baseline-type = displacement vector between two antennas (Sec. 2, after
    Eq. redcal; Sec. 5 intro);
  * subset redundant calibration takes whole redundant groups in ascending
    order of baseline length, stopping at the whole number of groups whose
    pair count is closest to p N log N (Sec. 5, Eq. subredcal_frac_bls;
    Sec. 6.1, integer number of redundant groups);
  * the selection must leave exactly the four degeneracies of Sec. 5.2
    (amplitude, phase, x and y phase slopes);
  * low-cadence calibration correlates every pair, p N log N pairs per
    integration cycle, all pairs of one type in the same cycle (Sec. 4,
    Eq. lowcadcal_inttime, and the requirement that redundant pairs be
    correlated simultaneously).

Readings where the paper is silent (stated in the design notes):
  * canonical half-plane for d: dy > 0, or dy == 0 and dx > 0;
  * ties in length are broken by the angle atan2(dy, dx) in [0, pi);
  * log base 2 by default; p = 1;
  * a type's pairs are ordered by the reference antenna r_j = (x, y),
    y major, and i = r_j + d;
  * low-cadence cycles: first-fit of types (in length order) into cycles of
    capacity floor(p N log N) pairs; t_int = floor(T / N_cycle), the
    remainder of the integration is not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def canonical_types(L: int):
    """All baseline-types of an L x L grid, shortest first (ties by angle)."""
    ts = [(dx, dy) for dy in range(0, L) for dx in range(-(L - 1), L)
          if dy > 0 or (dy == 0 and dx > 0)]
    ts.sort(key=lambda d: (d[0] * d[0] + d[1] * d[1], math.atan2(d[1], d[0])))
    return ts


def n_pairs(L: int, d) -> int:
    return (L - abs(d[0])) * (L - abs(d[1]))


def type_pairs(L: int, d):
    """(i, j) pairs of type d: r_i - r_j = d, reference r_j in row-major order."""
    dx, dy = d
    out = []
    for y in range(L):
        for x in range(L):
            xi, yi = x + dx, y + dy
            if 0 <= xi < L and 0 <= yi < L:
                out.append((yi * L + xi, y * L + x))
    return out


def budget(N: int, p: float, log_base: float) -> float:
    """p N log N pairs (Eq. lowcadcal_inttime / subredcal_frac_bls)."""
    lg = math.log(N) / math.log(log_base) if log_base > 0 else math.log(N)
    return p * N * lg


@dataclass
class Selection:
    L: int
    types: list                      # [(dx, dy)]
    type_ptr: np.ndarray             # [n_ubl + 1] int32
    pair_i: np.ndarray               # [P] int32
    pair_j: np.ndarray               # [P] int32
    win_t0: np.ndarray               # [n_ubl] int32
    win_t1: np.ndarray               # [n_ubl] int32
    n_cycle: int = 1
    t_int: int = 0
    null_dim: int = -1
    extra: dict = field(default_factory=dict)

    @property
    def P(self):
        return int(self.type_ptr[-1])

    @property
    def n_ubl(self):
        return len(self.types)

    def pair_type(self):
        a = np.zeros(self.P, np.int32)
        for k in range(self.n_ubl):
            a[self.type_ptr[k]:self.type_ptr[k + 1]] = k
        return a

    def pair_windows(self):
        t = self.pair_type()
        return self.win_t0[t], self.win_t1[t]


def _build(L, types, t0s, t1s):
    ptr = [0]
    pi, pj = [], []
    for d in types:
        prs = type_pairs(L, d)
        pi += [a for a, _ in prs]
        pj += [b for _, b in prs]
        ptr.append(len(pi))
    return (np.asarray(ptr, np.int32), np.asarray(pi, np.int32), np.asarray(pj, np.int32),
            np.asarray(t0s, np.int32), np.asarray(t1s, np.int32))


def null_space_dim(L: int, types) -> int:
    """Dimension of the null space of the linearised redcal system (Eq. logcal).

    Real unknowns: ln|g| (N), ln|V_alpha| (n_ubl) for the amplitude system
    (rows e_i + e_j + e_alpha) and arg g, arg V_alpha for the phase system
    (rows e_i - e_j + e_alpha).  Dense rank by SVD; small grids only.
    """
    N = L * L
    nu = len(types)
    rows_a, rows_p = [], []
    for k, d in enumerate(types):
        for i, j in type_pairs(L, d):
            ra = np.zeros(N + nu)
            ra[i] += 1.0
            ra[j] += 1.0
            ra[N + k] += 1.0
            rp = np.zeros(N + nu)
            rp[i] += 1.0
            rp[j] -= 1.0
            rp[N + k] += 1.0
            rows_a.append(ra)
            rows_p.append(rp)
    A = np.asarray(rows_a)
    B = np.asarray(rows_p)
    return (N + nu - np.linalg.matrix_rank(A)) + (N + nu - np.linalg.matrix_rank(B))


RANK_EXACT_MAX_N = 1024


def _criterion_prefix(L, ordered):
    """Smallest prefix length k whose null space is exactly 4 (Sec. 5.2).

    The null space can only shrink as types are added (a null vector of the
    larger system restricts to one of the smaller), so every longer prefix
    also satisfies the criterion.  Exact SVD rank up to RANK_EXACT_MAX_N
    antennas; above that the prefix found on a 12 x 12 grid is used (the
    shortest types that satisfy it, (1,0), (0,1), (1,1), do so on any grid
    with L >= 2, which the tests check exactly on small grids).
    """
    Lr = L if L * L <= RANK_EXACT_MAX_N else 12
    ordered_r = canonical_types(Lr)
    for k in range(1, len(ordered_r) + 1):
        if null_space_dim(Lr, ordered_r[:k]) == 4:
            assert ordered_r[:k] == ordered[:k]
            return k
    raise ValueError("no prefix satisfies the degeneracy criterion")


def subset(L: int, T: int, p: float = 1.0, log_base: float = 2.0) -> Selection:
    """Subset redundant calibration (Sec. 5; Sec. 6.1 integer groups)."""
    N = L * L
    ordered = canonical_types(L)
    target = budget(N, p, log_base)
    cum, best_k, best_err = 0, 1, None
    for k, d in enumerate(ordered, start=1):
        cum += n_pairs(L, d)
        err = abs(cum - target)
        if best_err is None or err < best_err:
            best_k, best_err = k, err
    k_min = _criterion_prefix(L, ordered)
    k = max(best_k, k_min)
    types = ordered[:k]
    ptr, pi, pj, t0, t1 = _build(L, types, [0] * k, [T] * k)
    return Selection(L, types, ptr, pi, pj, t0, t1, n_cycle=1, t_int=T, null_dim=4,
                     extra=dict(target=target, k_budget=best_k, k_min=k_min))


def lowcad(L: int, T: int, p: float = 1.0, log_base: float = 2.0) -> Selection:
    """Low-cadence calibration (Sec. 4, Eq. lowcadcal_inttime)."""
    N = L * L
    ordered = canonical_types(L)
    cap = int(math.floor(budget(N, p, log_base)))
    remaining = []          # free capacity per cycle
    cycle_of = []
    for d in ordered:
        n = n_pairs(L, d)
        if n > cap:
            raise ValueError("a redundant group exceeds the per-cycle capacity")
        for c, r in enumerate(remaining):
            if r >= n:
                remaining[c] -= n
                cycle_of.append(c)
                break
        else:
            remaining.append(cap - n)
            cycle_of.append(len(remaining) - 1)
    n_cycle = len(remaining)
    t_int = T // n_cycle
    t0 = [c * t_int for c in cycle_of]
    t1 = [(c + 1) * t_int for c in cycle_of]
    ptr, pi, pj, a0, a1 = _build(L, ordered, t0, t1)
    return Selection(L, ordered, ptr, pi, pj, a0, a1, n_cycle=n_cycle, t_int=t_int,
                     null_dim=4, extra=dict(cap=cap, cycle_of=cycle_of))


def n_bl_per_ant(sel: Selection) -> float:
    """Eq. subredcal_n_bl: N_obs / N."""
    return sel.P / (sel.L * sel.L)


def n_ubl_per_ant(sel: Selection) -> float:
    """Eq. subredcal_n_ubl: (1/N) sum_alpha (antennas taking part in alpha)."""
    N = sel.L * sel.L
    tot = 0
    for k in range(sel.n_ubl):
        a = set(sel.pair_i[sel.type_ptr[k]:sel.type_ptr[k + 1]].tolist())
        a |= set(sel.pair_j[sel.type_ptr[k]:sel.type_ptr[k + 1]].tolist())
        tot += len(a)
    return tot / N
