"""Write ``paper_1605_01800_gb300/cs_coexistence.json`` from the oracle's thermodynamics.

The table holds, for the Carnahan-Starling fluid with a = 1, b = 4, R = 1
(Eq. 15), the critical point and, at each reduced temperature the synthetic
workloads use, the Maxwell coexistence densities (Eq. 11), the spinodal
densities and the density where psi^2 of Eq. 13 turns negative. The input
generators read it to build initial density fields; it is written only by this
script, which calls nothing but ``oracle/``.

    python -m oracle.write_coexistence_table
"""
import json
import os
import warnings

from oracle import thermo

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1605_01800_gb300", "cs_coexistence.json")

A, B, R = 1.0, 4.0, 1.0


def reduced_temperatures():
    ts = {0.5, 0.55, 0.6, 0.7, 0.8, 0.9, 0.95}
    ts.update(round(0.5 + 0.45 * i / 31, 12) for i in range(32))
    return sorted(ts)


def main():
    warnings.simplefilter("ignore")
    Tc, rho_c, p_c = thermo.critical_point(A, B, R)
    rows = []
    for tr in reduced_temperatures():
        T = tr * Tc
        rg, rl, p0 = thermo.maxwell(T, A, B, R)
        sv, sl = thermo.spinodals(T, A, B, R)
        rows.append({"T_over_Tc": tr, "rho_g": rg, "rho_l": rl, "p0": p0,
                     "spinodal_vapour": sv, "spinodal_liquid": sl,
                     "psi_root": thermo.psi_root(T, A, B, R)})
    doc = {"eos": "Carnahan-Starling, Eq. 15", "a": A, "b": B, "R": R,
           "Tc": Tc, "rho_c": rho_c, "p_c": p_c,
           "written_by": "oracle/write_coexistence_table.py", "rows": rows}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=1)
    print(OUT, len(rows), "rows")


if __name__ == "__main__":
    main()
