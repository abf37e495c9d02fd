"""Residue -> balanced signed 8-bit limbs, by definition.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

The paper has no limbs: its experiments run over GF(2) and its base case is a
plain triple loop (Sec. 2.1, 2.2). The library's tensor-core form writes each
residue x in [0, p) as w signed 8-bit digits so that limb products can run on
the tensor cores exactly. The reading used by both sides:

* w = the least number of base-256 digits with 256^w >= p;
* representative r = x if x <= Hi, else x - p, where
  Hi = 127 * sum_{t<w} 256^t (the largest value w balanced digits reach), so r
  lies in [Lo, Hi] with Lo = -128 * sum_{t<w} 256^t, and r == x (mod p);
* digits d_0 .. d_{w-1} in [-128, 127], low digit first, with
  r = sum_t d_t 256^t: d_t is the balanced remainder of the running value
  modulo 256 (in [-128, 127]), and the running value is then (value - d_t)/256.

The product then satisfies A*B == sum_{s} 256^s * sum_{i+j=s} A_i B_j exactly
over the integers for the representatives, which is congruent to A*B mod p.
"""

from __future__ import annotations

import numpy as np


def n_limbs(p: int) -> int:
    w = 1
    while 256 ** w < p:
        w += 1
    return w


def bounds(w: int):
    s = sum(256 ** t for t in range(w))
    return -128 * s, 127 * s


def representative(x, p: int):
    """Representative r == x (mod p) in [Lo, Hi] (object or int64 array)."""
    w = n_limbs(p)
    _, hi = bounds(w)
    x = np.asarray(x, dtype=np.int64)
    return np.where(x <= hi, x, x - p)


def split(x, p: int) -> np.ndarray:
    """Limbs of residues x (any shape), as int8 with a new leading axis of size w."""
    w = n_limbs(p)
    r = representative(x, p).astype(np.int64)
    out = np.empty((w,) + r.shape, dtype=np.int8)
    v = r.copy()
    for t in range(w):
        d = ((v + 128) % 256) - 128          # balanced remainder in [-128, 127]
        out[t] = d.astype(np.int8)
        v = (v - d) // 256
    if np.any(v != 0):
        raise AssertionError("value outside the balanced range")
    return out


def recombine(limbs: np.ndarray) -> np.ndarray:
    """sum_t d_t 256^t as int64 (inverse of split on the representative)."""
    w = limbs.shape[0]
    r = np.zeros(limbs.shape[1:], dtype=np.int64)
    for t in reversed(range(w)):
        r = r * 256 + limbs[t].astype(np.int64)
    return r
