"""Write the stored expected values under tests/golden/.

Every number written here comes from ``oracle.exact`` (closed forms,
enumeration, transfer matrix, the exact finite-torus Ising partition function)
or is printed in the paper (cited beside it).  Nothing here calls the CUDA
library.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.exact as ex  # noqa: E402


def main():
    KC_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))

    # 1. Exact finite-torus Ising energy moments at beta_c (Kaufman 1949; the
    #    paper checks its q = 2 runs against this exact result, Sec. II.A).
    ising = {
        "citation": "Weigel arXiv:1105.5804 Sec. II.A (exactness check against the exact "
                    "finite-lattice Ising solution, Ferdinand & Fisher 1969); formula: Kaufman 1949",
        "convention": "H = -J sum sigma_i sigma_j, K = beta J = ln(1+sqrt2)/2; S = sum sigma_i sigma_j "
                      "over the 2N bonds; n_eq = (S + 2N)/2",
        "K": KC_ISING,
        "sizes": {},
    }
    for L in (4, 8, 16, 32, 64):
        S, varS = ex.ising_torus_energy_moments(L, KC_ISING)
        N = L * L
        ising["sizes"][str(L)] = {
            "mean_S": S,
            "var_S": varS,
            "mean_n_eq": (S + 2 * N) / 2.0,
            "var_n_eq": varS / 4.0,
            "energy_per_site": -S / N,
            "specific_heat_per_site": KC_ISING ** 2 * varS / N,
        }
    with open(os.path.join(HERE, "ising_exact_beta_c.json"), "w") as f:
        json.dump(ising, f, indent=1)

    # 1b. The same moments off criticality, at the beta / beta_c ratios of the
    #     paper's benchmark table (Sec. III, Table I: 0.6 and 1.4 for q = 2).
    off = {
        "citation": "Weigel arXiv:1105.5804 Table I (beta/beta_c = 0.6, 1.4 for q = 2); formula: Kaufman 1949",
        "convention": "as ising_exact_beta_c.json, with K = ratio * ln(1+sqrt2)/2",
        "L": 16,
        "ratios": {},
    }
    for ratio in (0.6, 1.4):
        K = ratio * KC_ISING
        S, varS = ex.ising_torus_energy_moments(16, K)
        off["ratios"][str(ratio)] = {"K": K, "mean_n_eq": (S + 2 * 256) / 2.0, "var_n_eq": varS / 4.0}
    with open(os.path.join(HERE, "ising_exact_off_critical.json"), "w") as f:
        json.dump(off, f, indent=1)

    # 2. Exact density of states of the q-state Potts model on the 4 x 4 torus.
    dos = {
        "citation": "Potts Hamiltonian, Weigel arXiv:1105.5804 Sec. II Eq. 1; row transfer matrix "
                    "count g(n_eq) of spin states with n_eq equal bonds on the periodic 4x4 torus",
        "g": {},
    }
    for q in (2, 3, 4):
        dos["g"][str(q)] = [int(v) for v in ex.potts_dos(4, 4, q)]
    with open(os.path.join(HERE, "potts_dos_4x4.json"), "w") as f:
        json.dump(dos, f, indent=1)

    # 3. Constants printed in the paper.
    consts = {
        "beta_c_potts_q2": {
            "value": math.log(1.0 + math.sqrt(2.0)),
            "expr": "ln(1+sqrt2)",
            "citation": "Weigel arXiv:1105.5804 Sec. II.B.3 (critical point of the q = 2 Potts model, "
                        "delta convention)",
        },
        "p_bond": {
            "expr": "p = 1 - exp(-beta J)",
            "citation": "Weigel arXiv:1105.5804 Sec. II, below Eq. 4, and Sec. II.A",
        },
    }
    with open(os.path.join(HERE, "paper_constants.json"), "w") as f:
        json.dump(consts, f, indent=1)


if __name__ == "__main__":
    main()
