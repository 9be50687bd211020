"""Matrix product operator of the Frenkel-Holstein Hamiltonian (Eq. holstein, Eq. mpo).

TEST INFRASTRUCTURE (oracle); see the package docstring.

H = sum_m E'_m n_m + sum_{m!=n} J_mn a_m^+ a_n + sum_{m,l} w_ml (b^+b [+ 1/2])
    + sum_{m,l} g_ml w_ml (b^+ + b) n_m,           E'_m = E_m - energy_offset.

Readings taken (the paper gives only Eq. holstein and Eq. mpo):
* the exciton operators act on a two-level site (|0>, |1>) as hard-core bosons
  with no Jordan-Wigner string; in the single-exciton sector this equals the
  fermionic form;
* a constant energy_offset is subtracted from every E_m and the zero-point term
  w/2 is optional (off by default).  Both shift H by a multiple of the conserved
  exciton number or by a constant, so populations are unchanged;
* the MPO is a finite-state automaton.  Channel 0 is "nothing placed yet",
  channel 1 "a whole term placed".  A cut with k electronic sites on its left and
  M-k on its right carries 2*min(k, M-k) hopping channels: while k <= M-k they
  are indexed by the left site m (a_m^+ or a_m pending), afterwards by the right
  site n (sum_m J_mn a_m^+ or sum_m J_nm a_m pending).  A cut inside the mode
  block of electronic site m carries one more channel, n_m pending a (b^+ + b).
"""
from __future__ import annotations

import numpy as np


def local_operators(kind: str, d: int):
    """Dense local operators in the site basis (|0>,|1>) or (|0>,...,|d-1>)."""
    if kind == "el":
        cr = np.array([[0.0, 0.0], [1.0, 0.0]])    # a^+ |0> = |1>
        return {"I": np.eye(2), "cr": cr, "an": cr.T.copy(), "n": np.diag([0.0, 1.0])}
    b = np.diag(np.sqrt(np.arange(1, d, dtype=float)), k=1)   # b |n> = sqrt(n) |n-1>
    return {"I": np.eye(d), "b": b, "bd": b.T.copy(), "x": b + b.T, "nb": np.diag(np.arange(d, dtype=float))}


def _cut_channels(k, M, in_block):
    """Channel labels of a cut: k electronic sites left, M-k right."""
    labels = [("idle",), ("done",)]
    if k <= M - k:
        for j in range(k):
            labels += [("Lcr", j), ("Lan", j)]
    else:
        for j in range(k, M):
            labels += [("Rcr", j), ("Ran", j)]
    if in_block:
        labels.append(("ph",))
    return labels


def build_mpo(p):
    """Site tensors W[i] with shape [W_left, W_right, d, d] (real float64).

    W[i][w, w', s', s] = <s'|op|s> for the operator that takes left channel w to
    right channel w'.  The left end selects channel "idle", the right end "done",
    so W[0] has one row and W[-1] one column.
    """
    chain = p.chain()
    M = p.n_el
    pos_of_el = {}     # electronic label -> index along the electronic order
    for j, m in enumerate(p.el_order):
        pos_of_el[m] = j
    d = p.phys_dims()
    N = len(chain)
    # channels of every cut 0..N (cut c lies left of site c)
    cuts = []
    for c in range(N + 1):
        k = sum(1 for kind, m, _ in chain[:c] if kind == "el")
        in_block = (0 < c < N and chain[c][0] == "vib")    # next site is a mode of the last el site
        cuts.append(_cut_channels(k, M, in_block))
    cuts[0] = [("idle",)]
    cuts[N] = [("done",)]
    Eoff = np.asarray(p.E, float) - p.energy_offset
    Jm = np.asarray(p.J, float)
    el_label = [m for m in p.el_order]
    W = []
    for i, (kind, m, kmode) in enumerate(chain):
        left, right = cuts[i], cuts[i + 1]
        li = {lab: a for a, lab in enumerate(left)}
        ri = {lab: a for a, lab in enumerate(right)}
        ops = local_operators(kind, d[i])
        T = np.zeros((len(left), len(right), d[i], d[i]))

        def put(lab_l, lab_r, op):
            if lab_l in li and lab_r in ri:
                T[li[lab_l], ri[lab_r]] += op

        put(("idle",), ("idle",), ops["I"])
        put(("done",), ("done",), ops["I"])
        if kind == "vib":
            w = float(p.omega[m][kmode])
            g = float(p.g[m][kmode])
            onsite = w * ops["nb"] + (0.5 * w * ops["I"] if p.include_zpe else 0.0)
            put(("idle",), ("done",), onsite)
            put(("ph",), ("done",), g * w * ops["x"])
            put(("ph",), ("ph",), ops["I"])
            for lab in left:                        # hopping channels pass through
                if lab[0] in ("Lcr", "Lan", "Rcr", "Ran"):
                    put(lab, lab, ops["I"])
        else:
            jm = pos_of_el[m]                       # index of this site along the electronic order
            put(("idle",), ("done",), Eoff[m] * ops["n"])
            put(("idle",), ("ph",), ops["n"])
            # complete terms whose right partner is this site
            for lab in left:
                if lab[0] == "Lcr":                 # a_src^+ pending -> J_{src,m} a_m
                    src = el_label[lab[1]]
                    put(lab, ("done",), Jm[src, m] * ops["an"])
                elif lab[0] == "Lan":               # a_src pending -> J_{m,src} a_m^+
                    src = el_label[lab[1]]
                    put(lab, ("done",), Jm[m, src] * ops["cr"])
                elif lab[0] == "Rcr" and lab[1] == jm:
                    put(lab, ("done",), ops["an"])
                elif lab[0] == "Ran" and lab[1] == jm:
                    put(lab, ("done",), ops["cr"])
            # open terms whose left partner is this site
            for lab in right:
                if lab[0] == "Lcr" and lab[1] == jm:
                    put(("idle",), lab, ops["cr"])
                elif lab[0] == "Lan" and lab[1] == jm:
                    put(("idle",), lab, ops["an"])
                elif lab[0] == "Rcr":               # J_{m,n} a_m^+ pending a_n
                    put(("idle",), lab, Jm[m, el_label[lab[1]]] * ops["cr"])
                elif lab[0] == "Ran":               # J_{n,m} a_m pending a_n^+
                    put(("idle",), lab, Jm[el_label[lab[1]], m] * ops["an"])
            # pass pending channels through this site
            for lab in left:
                if lab[0] in ("Lcr", "Lan") and lab[1] != jm:
                    if lab in ri:
                        put(lab, lab, ops["I"])
                    else:                           # switch to right-indexed channels
                        src = el_label[lab[1]]
                        for rl in right:
                            n = el_label[rl[1]] if rl[0] in ("Rcr", "Ran") else None
                            if lab[0] == "Lcr" and rl[0] == "Rcr":
                                put(lab, rl, Jm[src, n] * ops["I"])
                            elif lab[0] == "Lan" and rl[0] == "Ran":
                                put(lab, rl, Jm[n, src] * ops["I"])
                elif lab[0] in ("Rcr", "Ran") and lab[1] != jm:
                    put(lab, lab, ops["I"])
        W.append(T)
    return W


def mpo_to_dense(W):
    """Contract the MPO into a dense matrix on the full product basis (tiny chains only)."""
    acc = W[0][0]                                   # [W_r, s', s]
    acc = acc.reshape(acc.shape[0], acc.shape[1], acc.shape[2])
    for T in W[1:]:
        # acc[w, S', S] x T[w, w', s', s] -> [w', (S' s'), (S s)]
        new = np.einsum("wab,wvcd->vacbd", acc, T)
        acc = new.reshape(new.shape[0], new.shape[1] * new.shape[2], new.shape[3] * new.shape[4])
    return acc[0]
