"""Writes the stored expected values under tests/golden/ that are not printed in
the paper. Calls only the oracle (exact Riemann solver); run from the repo root:
    python tests/golden/gen_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import becker, riemann  # noqa: E402

SOD_LEFT = (1.0, 0.0, 1.0)
SOD_RIGHT = (0.125, 0.0, 0.1)


def main():
    L, R = riemann.State(*SOD_LEFT), riemann.State(*SOD_RIGHT)
    st = riemann.solve_star(L, R, 1.4)
    out = {
        "_source": "oracle/riemann.py exact Riemann solution, gamma = 1.4, Sod states of Sec. 3.1",
        "p_star": st.p, "u_star": st.u, "rho_star_L": st.rho_L, "rho_star_R": st.rho_R,
        "shock_speed": st.sR_head, "fan_head": st.sL_head, "fan_tail": st.sL_tail,
        "lambda_max": riemann.max_signal_speed(L, R, 1.4),
        "shock_position_t0.2": riemann.shock_position(L, R, 0.2, 0.5, 1.4),
    }
    with open(os.path.join(HERE, "sod_exact.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out, indent=1))
    b = becker.paper_case()
    rho2, u2_lab, p2 = b.downstream()
    bk = {
        "_source": "oracle/becker.py exact Becker profile, gamma 1.4, Pr 3/4, mu 2e-3, M_s 2, "
                   "upstream (rho, c) = (1, 1) (Sec. 3.1)",
        "u1": b.u1, "u2": b.u2, "rho2": rho2, "u2_lab": u2_lab, "p2": p2,
        "lambda_max": b.max_signal_speed(),
        "w_max_slope_rho": b.thickness(),
    }
    with open(os.path.join(HERE, "becker_exact.json"), "w") as fh:
        json.dump(bk, fh, indent=1)
        fh.write("\n")
    print(json.dumps(bk, indent=1))


if __name__ == "__main__":
    main()
