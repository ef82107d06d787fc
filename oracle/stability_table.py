"""Prints the stability diagram of the scheme (spectral radius of one step's
amplification matrix against Omega = tau sqrt(lambda), Sec. 3.2) as a markdown table,
for the orders 2k = 2, 4 and rho_inf in {0, 0.5, 0.8, 1}. Test infrastructure: it calls
only the oracle.

Usage: python -m oracle.stability_table
"""
import math

import oracle


def main():
    rhos = (0.0, 0.5, 0.8, 1.0)
    omegas = (0.01, 0.1, 0.5, 1.0, 1.5)
    print("| Omega | " + " | ".join("k=%d, rho=%g" % (k, r) for k in (1, 2) for r in rhos) + " |")
    print("|---|" + "---|" * (2 * len(rhos)))
    rows = list(omegas) + ["limit"]
    for om in rows:
        cells = []
        for k in (1, 2):
            for r in rhos:
                o = math.sqrt(oracle.theta_crit(r)) * 0.999 if om == "limit" else om
                cells.append("%.6f" % oracle.spectral_radius(k, r, o))
        print("| %s | %s |" % (om if om != "limit" else "0.999 sqrt(Theta_crit)", " | ".join(cells)))
    print()
    print("sqrt(Theta_crit): " + ", ".join("rho=%g: %.4f" % (r, math.sqrt(oracle.theta_crit(r))) for r in rhos))


if __name__ == "__main__":
    main()
