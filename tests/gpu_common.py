"""Shared helpers of the GPU tests: contexts, oracle models and error bounds."""
from __future__ import annotations

import json
import os

import numpy as np

from oracle import hamiltonian as H

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U32 = 2.0 ** -24     # unit roundoff, fp32
U64 = 2.0 ** -53     # unit roundoff, fp64


def golden():
    return json.load(open(os.path.join(GOLD, "oracle_values.json")))


def device_ctx(w, basis=None, nf=None):
    """Context on cuda:0 with the workload's Hamiltonian and either the given
    basis words or the library's sampled basis of size nf (default w.n_f)."""
    import paper_2509_22975_gb300 as pkg
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up, w.n_dn)
    if basis is not None:
        ctx.mcd_set_basis(basis)
    else:
        ctx.mcd_build_basis(w.seed, nf or w.n_f, w.beta, [w.seed_word()])
    return ctx


def model(w):
    return H.Model(w.n_sites, w.lat.t, w.eps, w.U_sites)


def row_terms_bound(n_bonds: int) -> int:
    """Upper bound on the number of terms summed in one row (diagonal + one
    hop per bond and spin) plus the roundings outside the sum."""
    return 2 * n_bonds + 4


def apply_bound(absHx, n_terms: int, u: float):
    """|y_computed - y_exact| <= n_terms * u * (|H~| |x|), the standard bound of
    a recursively summed dot product (each of n_terms products and partial
    sums rounded once) with unit roundoff u."""
    return n_terms * u * absHx
