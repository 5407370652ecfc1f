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


# --------------------------------------------------------------------------- lattice layouts
# Arrays on a lattice that is not fully occupied -- the paper's own arrays
# are hexagonal (Sec. 3) -- are held as an L x L bounding grid of lattice
# points (index i = y L + x) with a mask of the occupied points.  Lattice
# "square": unit spacing; "triangular": basis (1, 0), (1/2, sqrt(3)/2), so a
# type (dx, dy) has squared length dx^2 + dx dy + dy^2 and physical angle
# atan2(dy sqrt(3)/2, dx + dy/2).  The canonical half-plane rule
# (dy > 0, or dy == 0 and dx > 0) is the same on both lattices.

def hex_mask(s: int):
    """Hexagonal array of side s (3 s (s - 1) + 1 antennas) on a triangular
    lattice: axial coordinates (a, b) with |a|, |b|, |a + b| <= s - 1, held in
    the (2 s - 1)^2 bounding grid at x = a + s - 1, y = b + s - 1.  Returns
    (L, mask[L * L] uint8)."""
    L = 2 * s - 1
    m = np.zeros(L * L, np.uint8)
    for y in range(L):
        for x in range(L):
            if s - 1 <= x + y <= 3 * s - 3:
                m[y * L + x] = 1
    return L, m


def type_length2(d, lattice: str):
    dx, dy = d
    return dx * dx + dx * dy + dy * dy if lattice == "triangular" else dx * dx + dy * dy


def type_angle(d, lattice: str):
    dx, dy = d
    if lattice == "triangular":
        return math.atan2(dy * math.sqrt(3.0) / 2.0, dx + dy / 2.0)
    return math.atan2(dy, dx)


def masked_type_pairs(L: int, mask, d):
    """(i, j) pairs of type d between occupied points, r_j row-major."""
    return [(i, j) for i, j in type_pairs(L, d) if mask[i] and mask[j]]


def layout_types(L: int, mask, lattice: str):
    """Baseline-types with at least one occupied pair, shortest first (ties
    by physical angle), with their pair counts."""
    ts = [d for d in canonical_types(L) if masked_type_pairs(L, mask, d)]
    ts.sort(key=lambda d: (type_length2(d, lattice), type_angle(d, lattice)))
    return ts, [len(masked_type_pairs(L, mask, d)) for d in ts]


def masked_null_space_dim(L: int, mask, types) -> int:
    """null_space_dim over the occupied antennas only (dense SVD rank)."""
    occ = np.flatnonzero(np.asarray(mask))
    col = {int(a): c for c, a in enumerate(occ)}
    N, nu = len(occ), len(types)
    rows_a, rows_p = [], []
    for k, d in enumerate(types):
        for i, j in masked_type_pairs(L, mask, d):
            ra = np.zeros(N + nu)
            ra[col[i]] += 1.0
            ra[col[j]] += 1.0
            ra[N + k] += 1.0
            rp = np.zeros(N + nu)
            rp[col[i]] += 1.0
            rp[col[j]] -= 1.0
            rp[N + k] += 1.0
            rows_a.append(ra)
            rows_p.append(rp)
    A = np.asarray(rows_a)
    B = np.asarray(rows_p)
    return (N + nu - np.linalg.matrix_rank(A)) + (N + nu - np.linalg.matrix_rank(B))


def subset_layout(L: int, mask, lattice: str, T: int, p: float = 1.0, log_base: float = 2.0) -> Selection:
    """Subset redundant calibration (Sec. 5) on a masked lattice: whole types
    in ascending physical length until the pair count is the whole number of
    groups closest to p N log N (N = occupied antennas), extended if needed
    until exactly four degeneracies remain (Sec. 5.2, exact SVD rank)."""
    mask = np.asarray(mask, np.uint8)
    N = int(mask.sum())
    ordered, counts = layout_types(L, mask, lattice)
    target = budget(N, p, log_base)
    cum, best_k, best_err = 0, 1, None
    for k, n in enumerate(counts, start=1):
        cum += n
        err = abs(cum - target)
        if best_err is None or err < best_err:
            best_k, best_err = k, err
    k = best_k
    while masked_null_space_dim(L, mask, ordered[:k]) != 4:
        k += 1
    types = ordered[:k]
    ptr, pi, pj = [0], [], []
    for d in types:
        prs = masked_type_pairs(L, mask, d)
        pi += [a for a, _ in prs]
        pj += [b for _, b in prs]
        ptr.append(len(pi))
    return Selection(L, types, np.asarray(ptr, np.int32), np.asarray(pi, np.int32), np.asarray(pj, np.int32),
                     np.zeros(k, np.int32), np.full(k, T, np.int32), n_cycle=1, t_int=T, null_dim=4,
                     extra=dict(target=target, k_budget=best_k, mask=mask, lattice=lattice, N=N))


def compact(sel: Selection, mask):
    """Pairs and lattice coordinates in the occupied-antenna numbering:
    (pair_i, pair_j, pos [N_occ x 2]) for the oracle's calibration."""
    occ = np.flatnonzero(np.asarray(mask))
    col = -np.ones(len(mask), np.int64)
    col[occ] = np.arange(len(occ))
    pos = np.stack([occ % sel.L, occ // sel.L], 1).astype(float)
    return col[sel.pair_i], col[sel.pair_j], pos


def lowcad_layout(L: int, mask, lattice: str, T: int, p: float = 1.0, log_base: float = 2.0) -> Selection:
    """Low-cadence calibration (Sec. 4) on a masked lattice: every type with
    an occupied pair, first-fit into cycles of floor(p N log N) pairs (N the
    occupied points), t_int = floor(T / N_cycle)."""
    mask = np.asarray(mask, np.uint8)
    N = int(mask.sum())
    ordered, counts = layout_types(L, mask, lattice)
    cap = int(math.floor(budget(N, p, log_base)))
    remaining, cycle_of = [], []
    for n in counts:
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
    ptr, pi, pj = [0], [], []
    for d in ordered:
        prs = masked_type_pairs(L, mask, d)
        pi += [a for a, _ in prs]
        pj += [b for _, b in prs]
        ptr.append(len(pi))
    t0 = [c * t_int for c in cycle_of]
    t1 = [(c + 1) * t_int for c in cycle_of]
    return Selection(L, ordered, np.asarray(ptr, np.int32), np.asarray(pi, np.int32), np.asarray(pj, np.int32),
                     np.asarray(t0, np.int32), np.asarray(t1, np.int32), n_cycle=n_cycle, t_int=t_int,
                     null_dim=4, extra=dict(cap=cap, cycle_of=cycle_of, mask=mask, lattice=lattice, N=N))
