"""Test helpers: conversion between the library's block layout of a two-site wavefunction
and the oracle's dense (l, s1, s2, r) arrays, and problem set-up shared by GPU tests."""
import numpy as np


def _offsets(bond):
    return np.cumsum([0] + [m for (_, _, m) in bond])


def layout_to_dense(x, table, bond_l, bond_r):
    """Flat block-layout vector -> dense (M_l, 4, 4, M_r) array (zeros elsewhere)."""
    ol, orr = _offsets(bond_l), _offsets(bond_r)
    d = np.zeros((ol[-1], 4, 4, orr[-1]))
    for jl, s1, s2, jr, off, size in table:
        ml, mr = bond_l[jl][2], bond_r[jr][2]
        d[ol[jl]:ol[jl] + ml, s1, s2, orr[jr]:orr[jr] + mr] = x[off:off + size].reshape(ml, mr)
    return d


def dense_to_layout(d, table, bond_l, bond_r):
    """Dense (M_l, 4, 4, M_r) array -> flat block-layout vector."""
    ol, orr = _offsets(bond_l), _offsets(bond_r)
    n = int(sum(t[5] for t in table))
    x = np.zeros(n)
    for jl, s1, s2, jr, off, size in table:
        ml, mr = bond_l[jl][2], bond_r[jr][2]
        x[off:off + size] = d[ol[jl]:ol[jl] + ml, s1, s2, orr[jr]:orr[jr] + mr].ravel()
    return x


def layout_mask(table, bond_l, bond_r):
    return layout_to_dense(np.ones(int(sum(t[5] for t in table))), table, bond_l, bond_r) != 0
