"""Derive the Cr-Cr / Cr-C parameter set used by every workload and write it as JSON.

The paper prints the functional forms of its potentials (Appendix, Eqs. A2-A5) but
not their parameters (they come from its refs. [42] and [34]); only d = 1.65 (Eq. A4)
and r_e = 2.754 A (Sec. 2.6) are given.  This script fixes a self-consistent set,
"derived for this implementation, not the paper's values":

  * f_e = 1, beta = 6, n = 0.75, F_o = 2.74 eV (chosen);
  * one cut-off rc = d r_e for f, f^2 and Phi, with the shifted-force form of f;
  * rho_e, P_e = the lattice sums of f and f^2 in perfect BCC at a = 2.885 A, so that
    F'(rho_e) = M'(P_e) = M(P_e) = 0 at equilibrium;
  * a0..a3 and alpha from five linear conditions on the BCC lattice energy per atom:
      dE/da = 0 at a = 2.885 A, E = -E_c (4.10 eV),
      C' = (C11 - C12)/2 = 25 GPa, C44 = 99.0 GPa, B = 152.3 GPa
    (room-temperature Cr has C44 = 99.0 GPa and B = 152.3 GPa, but C' = 140.6 GPa: with
    that C' the fitted cubic of Eq. A4 develops a 1 eV deep well near 3.5 A and the BCC
    lattice is only metastable -- an MD run at 300 K leaves it and heats to thousands of
    kelvin.  C' = 25 GPa is the largest of the values tried whose lattice stays solid
    at 300-600 K, so that is the target; the lattice energy
    is linear in (a0..a3, F_o, alpha), so each condition is a linear row whose
    coefficients are lattice sums evaluated with the oracle's own potential functions
    (unit coefficients), second derivatives by central differences in the strain;
  * Morse placeholders D_o = 0.2 eV, alpha_x = 6, y_eq = 2.2 A, rc_m = 6 A.
  * --indentation: the same Cr-Cr set with a Cr-C reading for the indentation run of
    Sec. 4.3 (also derived, not the paper's): alpha_x = 10, D_o = 0.02 eV (y_eq, rc_m as
    above).  With the placeholders' long soft tail (alpha_x = 6, D_o = 0.2 eV) the film wets
    the tip and the load stays adhesive over the whole protocol, so neither the Hertz law
    nor the Oliver-Pharr analysis applies.  A scan of the full protocol on the paper's 11k
    system (alpha_x 6/8/10, D_o 0.02-0.2 eV) gave the least adhesion on loading with
    alpha_x = 10, D_o = 0.02 eV: the load dips to -0.7 eV/A before contact and peaks at
    +15 eV/A (the paper's 27.4 eV/A is out of reach of any Cr-C reading here: the derived
    film is softer than Cr, C' = 25 GPa).

Run:  python oracle/derive_params.py   (writes paper_1507_07068_gb300/cr_c_params.json)
      python oracle/derive_params.py --rc 8.262 --out paper_1507_07068_gb300/cr_c_params_rstar.json
      (the same fit with the paper's long cut-off r* = 3 r_e = 8.262 A for f and f^2,
      Sec. 2.6; Phi still ends at its double root d r_e)
      python oracle/derive_params.py --indentation --out paper_1507_07068_gb300/cr_c_params_indent.json
Only oracle/ is called.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402

GPA = 160.21766208  # 1 eV/A^3 in GPa

CHOSEN = dict(r_e=2.754, f_e=1.0, beta=6.0, n=0.75, F_o=2.74, d=1.65,
              D_o=0.2, alpha_x=6.0, y_eq=2.2, rc_m=6.0, shifted=1, tabulated=1,
              r_min=1.0, h=1e-3)
TARGET = dict(a_lat=2.885, E_c=4.10, C_prime=25.0, C44=99.0, B=152.3)


def bcc_vectors(a: float, rmax: float) -> np.ndarray:
    m = int(np.ceil(rmax / a)) + 1
    g = np.arange(-m, m + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    c = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(float)
    v = np.concatenate([c, c + 0.5]) * a
    r = np.sqrt((v * v).sum(1))
    return v[(r > 1e-9) & (r < rmax + 0.5)]


def base_params(**kw) -> dict:
    p = dict(CHOSEN)
    p.update(rc=p["d"] * p["r_e"], rho_e=1.0, P_e=1.0, alpha=0.0, a0=0.0, a1=0.0, a2=0.0, a3=0.0)
    p.update(kw)
    return p


INDENTATION_MORSE = dict(D_o=0.02, alpha_x=10.0)


def main(out_path: str | None = None, rc: float | None = None, indentation: bool = False) -> dict:
    a = TARGET["a_lat"]
    p0 = base_params(tabulated=0) if rc is None else base_params(tabulated=0, rc=rc)
    rc = p0["rc"]
    V = bcc_vectors(a, rc)
    omega = a ** 3 / 2.0
    pot_f = oracle.Potential(p0)

    def dens(strain):
        r = np.sqrt(((V @ (np.eye(3) + strain).T) ** 2).sum(1))
        f, _ = pot_f.evalv(oracle.OR_F, r)
        return f.sum(), (f * f).sum(), r

    rho_e, P_e, _ = dens(np.zeros((3, 3)))

    def unit_pots():
        pots = []
        for k in range(4):
            pots.append(oracle.Potential(base_params(tabulated=0, rc=rc, rho_e=rho_e, P_e=P_e, **{f"a{k}": 1.0})))
        pots.append(oracle.Potential(base_params(tabulated=0, rc=rc, rho_e=rho_e, P_e=P_e, F_o=1.0)))
        pots.append(oracle.Potential(base_params(tabulated=0, rc=rc, rho_e=rho_e, P_e=P_e, F_o=0.0, alpha=1.0)))
        return pots

    pots = unit_pots()

    def energy_terms(strain):
        """per-atom lattice energy for unit (a0, a1, a2, a3, F_o, alpha)"""
        rho, P, r = dens(strain)
        row = []
        for k in range(4):
            phi, _ = pots[k].evalv(oracle.OR_PHI, r)
            row.append(0.5 * phi.sum())
        row.append(pots[4].eval(oracle.OR_EMBED, rho)[0])
        row.append(pots[5].eval(oracle.OR_MTERM, P)[0])
        return np.array(row)

    def second(strain_of):
        e = 1e-4
        return (energy_terms(strain_of(e)) + energy_terms(strain_of(-e)) - 2 * energy_terms(strain_of(0.0))) / e ** 2

    # equilibrium: dE/de for hydrostatic strain = 0.5 sum Phi'(r) r  (F'(rho_e) = M'(P_e) = 0)
    _, _, r0 = dens(np.zeros((3, 3)))
    eq = []
    for k in range(4):
        _, dphi = pots[k].evalv(oracle.OR_PHI, r0)
        eq.append(0.5 * (dphi * r0).sum())
    eq += [0.0, 0.0]
    coh = energy_terms(np.zeros((3, 3)))
    cp = second(lambda e: np.diag([e, -e, 0.0])) / (4.0 * omega) * GPA

    def shear(e):
        s = np.zeros((3, 3)); s[0, 1] = s[1, 0] = 0.5 * e
        return s
    c44 = second(shear) / omega * GPA
    bulk = second(lambda e: np.eye(3) * e) / (9.0 * omega) * GPA

    F_o = CHOSEN["F_o"]
    A = np.array([eq, coh, cp, c44, bulk])
    rhs = np.array([0.0, -TARGET["E_c"], TARGET["C_prime"], TARGET["C44"], TARGET["B"]])
    # unknowns (a0, a1, a2, a3, alpha); F_o fixed
    rhs = rhs - A[:, 4] * F_o
    M = A[:, [0, 1, 2, 3, 5]]
    sol = np.linalg.solve(M, rhs)
    params = base_params(rc=rc, rho_e=float(rho_e), P_e=float(P_e), a0=float(sol[0]), a1=float(sol[1]),
                         a2=float(sol[2]), a3=float(sol[3]), alpha=float(sol[4]), F_o=F_o)
    params["_note"] = ("derived for this implementation, not the paper's values: the paper's refs. [42] "
                       "and [34] are not printed; see oracle/derive_params.py")
    params["_targets"] = TARGET
    if indentation:
        params.update(INDENTATION_MORSE)
        params["_note"] += ("; Cr-C reading for the indentation run (alpha_x = 10, D_o = 0.02 eV): the "
                            "least adhesive contact of a scan of the paper's 11k-system protocol")
    if out_path is None:
        out_path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "paper_1507_07068_gb300", "cr_c_params.json")
    with open(out_path, "w") as fh:
        json.dump(params, fh, indent=1, sort_keys=True)
        fh.write("\n")
    return params


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--rc", type=float, default=None, help="cut-off of f and f^2 (A); default d r_e")
    ap.add_argument("--out", default=None)
    ap.add_argument("--indentation", action="store_true", help="the Cr-C reading of the indentation run")
    a = ap.parse_args()
    print(json.dumps(main(a.out, a.rc, a.indentation), indent=1, sort_keys=True))
