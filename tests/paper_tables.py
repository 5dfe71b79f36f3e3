"""The paper's printed errors of the diagonal translation (tests/golden/translation_e_phi.json)
and of the interface extension (tests/golden/extension_e_phi.json), and the error measure
they use; shared by the oracle and GPU table tests."""
import json
import os

import numpy as np

from paper_2007_07760_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "translation_e_phi.json")
GOLDEN_EXT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "extension_e_phi.json")
SCHEMES = {"T2S2CD": (2, 1, 2), "T2S3": (3, 0, 2), "T3S3": (3, 0, 3)}   # order, flux, stages


def paper_value(scheme: str, cfl: float, n: int) -> float:
    t = json.load(open(GOLDEN))
    return t["E_phi"][scheme][str(cfl)][t["N"].index(n)]


def problem(scheme: str, cfl: float, n: int):
    order, flux, stages = SCHEMES[scheme]
    return WL.translation(n, order, flux, stages, cfl)


def e_phi(phi: np.ndarray, phi0: np.ndarray) -> float:
    """L2-norm error of phi against the initial field (the measure of Sec. III)."""
    return float(np.sqrt(((phi - phi0) ** 2).sum() / (phi0 ** 2).sum()))


def extension_entries():
    """Every printed DUGKS entry of the extension table: (scheme, cfl, Pe, E_phi)."""
    t = json.load(open(GOLDEN_EXT))
    return [(sch, float(c), pe, row[i]) for sch, rows in t["E_phi"].items() for c, row in rows.items()
            for i, pe in enumerate(t["Pe"])]
