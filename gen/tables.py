"""Seeded binding tables for the pairwise-join workloads.

A binding table is a list of variable ids and one uint32 column per variable
(structure of arrays), the shape of a triple pattern's partial-match table in
Table 1 of the paper.  Nothing here joins anything.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import Rng, mix64, zipf_ranks


@dataclass
class Table:
    """Plain container: ``vars[c]`` is the variable id of column ``cols[c]``."""

    vars: list
    cols: list = field(default_factory=list)

    @property
    def nrows(self) -> int:
        return int(self.cols[0].shape[0]) if self.cols else self._nrows

    _nrows: int = 0

    @staticmethod
    def unit(nrows: int = 1) -> "Table":
        t = Table([], [])
        t._nrows = nrows
        return t


def pairwise_uniform(seed: int = 1, n_left: int = 16384, n_right: int = 8192,
                     key_domain: int = 4096, value_domain: int = 1 << 20):
    """Single pairwise join, uniform keys: Tp1(key, v1) and Tp2(key, v2).

    Variable ids: key = 0, v1 = 1, v2 = 2.
    """
    rng = Rng(seed, 0)
    lk = rng.below(n_left, key_domain).astype(np.uint32)
    lv = rng.below(n_left, value_domain).astype(np.uint32)
    rk = rng.below(n_right, key_domain).astype(np.uint32)
    rv = rng.below(n_right, value_domain).astype(np.uint32)
    return Table([0, 1], [lk, lv]), Table([0, 2], [rk, rv])


def key_pair_bijection(ids: np.ndarray, seed: int):
    """Map distinct key ids to distinct (x, y) uint32 pairs via a 64-bit bijection."""
    salt = np.uint64(int(mix64(np.uint64(seed ^ 0xA5A5A5A5))))
    z = mix64(ids.astype(np.uint64) ^ salt)
    return (z >> np.uint64(32)).astype(np.uint32), (z & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def skewed_two_key(seed: int = 3, log_a: int = 26, log_b: int = 24, log_keys: int = 22,
                   s: float = 1.1, reps: int = 4):
    """Large join on two shared variables (x, y).

    A: 2^log_a rows (x, y, a1, a2); its key ids follow Zipf(s) over 2^log_keys ids,
    rank -> id through a seeded permutation.  B: 2^log_b rows (x, y, b1, b2) holding
    every key id exactly ``reps`` times in shuffled order (log_b = log_keys + log2(reps)),
    so the join has exactly reps * 2^log_a rows.  Variable ids: x=0, y=1, a1=2, a2=3,
    b1=4, b2=5.
    """
    nk = 1 << log_keys
    assert (1 << log_b) == nk * reps
    rng = Rng(seed, 0)
    perm = rng.permutation(nk)
    a_ids = perm[zipf_ranks(Rng(seed, 1), 1 << log_a, nk, s)]
    ax, ay = key_pair_bijection(a_ids, seed)
    ra = Rng(seed, 2)
    a1, a2 = ra.u32(1 << log_a), ra.u32(1 << log_a)
    b_ids = Rng(seed, 3).permutation(1 << log_b) // reps
    bx, by = key_pair_bijection(b_ids, seed)
    rb = Rng(seed, 4)
    b1, b2 = rb.u32(1 << log_b), rb.u32(1 << log_b)
    return Table([0, 1, 2, 3], [ax, ay, a1, a2]), Table([0, 1, 4, 5], [bx, by, b1, b2])


_AFFINE_PRIME = 4294967291  # largest prime below 2^32; coprime to every smaller domain


def uneven_batch(seed: int = 4, n_joins: int = 256, log_lo: float = 8.0, log_hi: float = 22.0):
    """Batch of independent joins of uneven size.

    Per join: rows per side floor(2^U[log_lo, log_hi]); 2-4 columns per side with the
    key in column 0 (variable 0); key domain D = max(64, ceil(|R|/2)); left keys Zipf(s)
    over D with s drawn from {0, 0.8, 1.2} (rank -> id through a seeded affine bijection
    mod D), right keys uniform over D.  Non-key columns are uniform uint32 with fresh
    variable ids (left 1.., right 10..).
    Returns a list of (L, R, s) triples.
    """
    out = []
    for j in range(n_joins):
        r = Rng(seed, 1000 + j)
        e_l, e_r = log_lo + (log_hi - log_lo) * r.unit(2)
        nl, nr = int(2.0 ** e_l), int(2.0 ** e_r)
        cl, cr = (int(v) for v in r.between(2, 2, 4))
        s = (0.0, 0.8, 1.2)[int(r.below(1, 3)[0])]
        d = max(64, -(-nr // 2))
        a = _AFFINE_PRIME % d or 1
        while np.gcd(a, d) != 1:
            a += 1
        b = int(r.below(1, d)[0])
        lk = ((zipf_ranks(r, nl, d, s) * a + b) % d).astype(np.uint32)
        rk = r.below(nr, d).astype(np.uint32)
        L = Table([0] + list(range(1, cl)), [lk] + [r.u32(nl) for _ in range(cl - 1)])
        R = Table([0] + list(range(10, 10 + cr - 1)), [rk] + [r.u32(nr) for _ in range(cr - 1)])
        out.append((L, R, s))
    return out


def random_table(rng: Rng, nrows: int, vars_: list, domain: int) -> Table:
    """Small random table, every column uniform over [0, domain)."""
    return Table(list(vars_), [rng.below(nrows, domain).astype(np.uint32) for _ in vars_])
