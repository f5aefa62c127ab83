"""The test densities of the paper's Sec. 5 with their exact potentials, on the box
[-2, 2]^3 of Tables 1, 3, 5 and 7 (the bump and oscillating densities re-derived as
-Laplace of their stated solutions).  Shared by the oracle pins and the GPU tables test."""
import json
import os

import numpy as np

from oracle import exact
from paper_1612_01799_gb300 import densities as D

HERE = os.path.dirname(os.path.abspath(__file__))
BOX_L = 2.0


def load_cases():
    with open(os.path.join(HERE, "golden", "paper_tables.json")) as f:
        return json.load(f)["cases"]


def radius(N, L, c=(0.0, 0.0, 0.0)):
    x = D.axis(N, L)
    return np.sqrt((x[None, None, :] - c[0]) ** 2 + (x[None, :, None] - c[1]) ** 2
                   + (x[:, None, None] - c[2]) ** 2)


def paper_case(case, N):
    """(rho, exact u) of one table case at N points per axis."""
    L = BOX_L
    r = radius(N, L)
    if case["density"] == "gaussian":
        return D.gaussian_iso(N, L, case["sigma"]), exact.gaussian_iso(r, case["sigma"])
    if case["density"] == "two_gaussians":
        d = np.array(case["d"])
        rho = D.paper_two_gaussians(N, [-L] * 3, [L] * 3, d=d, s1=case["sigma1"], s2=case["sigma2"])
        ue = 0.5 * (exact.gaussian_iso(radius(N, L, d), case["sigma1"])
                    + exact.gaussian_iso(radius(N, L, -d), case["sigma2"]))
        return rho, ue
    x = D.axis(N, L)
    if case["density"] == "aniso":
        sg = case["sigma"]
        return D.paper_aniso(N, L, sg), exact.aniso_exp(x[None, None, :], x[None, :, None],
                                                        x[:, None, None], (0, 0, 0), sg)
    if case["density"] == "oscillating":
        return (D.paper_oscillating(N, L, case["sigma"], case["omega"]),
                exact.oscillating(r, case["sigma"], case["omega"]))
    raise KeyError(case["density"])
