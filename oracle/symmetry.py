"""Matrices at a reducible q from the irreducible one by a rotation (oracle), Sec. 3.1, Eq. symeps.

TEST INFRASTRUCTURE ONLY (see the package header).

Eq. symeps: eps^-1_{G,G'}(q, w) = eps^-1_{S^-1(G+D), S^-1(G'+D')}(q*, w) e^{-i(G-G').T}, with q the
image of the irreducible q* under the rotation and D the rewind vector that brings it back to the
first zone.  Written for fractional row vectors with the integer matrix S of the rotation
(S acts as k -> k S): q* S = q + G_s, and then q + G = (q* + G*) S for G = G* S + G_s, so
    X_{G,G'}(q) = X_{G*,G'*}(q*)
for chi0, eps^-1 and W alike (|q+G| = |q*+G*|: the Coulomb factors agree).  The crystals of this
path are symmorphic (no fractional translation T), so there is no phase.
Reading: the primed rewind vector of the printed equation is the same vector as the unprimed one
(both G and G' belong to the same q).
"""
import numpy as np


def image_index(G_irr, G, S, g_s):
    """perm[g] = index in G_irr of G* with G[g] = G* S + g_s (raises if the spheres do not match)."""
    G_irr = np.asarray(G_irr, dtype=np.int64)
    G = np.asarray(G, dtype=np.int64)
    mapped = G_irr @ np.asarray(S, dtype=np.int64) + np.asarray(g_s, dtype=np.int64)[None, :]
    pos = {tuple(r): i for i, r in enumerate(mapped)}
    perm = np.array([pos.get(tuple(r), -1) for r in G])
    if len(G) != len(G_irr) or np.any(perm < 0):
        raise ValueError("the rotation does not map the sphere of q* onto the sphere of q")
    return perm


def rotate(X_irr, perm):
    """X(q)[f, g, g'] = X(q*)[f, perm[g], perm[g']]."""
    return np.asarray(X_irr)[:, perm][:, :, perm]
