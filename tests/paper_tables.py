"""The paper's printed errors of the diagonal translation (tests/golden/translation_e_phi.json),
the interface extension (tests/golden/extension_e_phi.json), Zalesak's disk
(tests/golden/zalesak_e_phi.json) and the smoothed deformation
(tests/golden/deformation_e_phi.json), and the error measure they use; shared by the
oracle and GPU table tests."""
import dataclasses
import json
import os

import numpy as np

from paper_2007_07760_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "translation_e_phi.json")
GOLDEN_EXT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "extension_e_phi.json")
SCHEMES = {"T2S2CD": (2, 1, 2), "T2S3": (3, 0, 2), "T3S3": (3, 0, 3), "T2S5": (5, 0, 2)}   # order, flux, stages


def paper_value(scheme: str, cfl: float, n: int) -> float:
    t = json.load(open(GOLDEN))
    return t["E_phi"][scheme][str(cfl)][t["N"].index(n)]


def problem(scheme: str, cfl: float, n: int):
    order, flux, stages = SCHEMES[scheme]
    return WL.translation(n, order, flux, stages, cfl)


def e_phi(phi: np.ndarray, phi0: np.ndarray) -> float:
    """L2-norm error of phi against the initial field (the measure of Sec. III)."""
    return float(np.sqrt(((phi - phi0) ** 2).sum() / (phi0 ** 2).sum()))


def extension_entries(schemes=("T2S2CD", "T2S3", "T3S3")):
    """The printed DUGKS entries of the extension table of the given schemes:
    (scheme, cfl, Pe, E_phi)."""
    t = json.load(open(GOLDEN_EXT))
    return [(sch, float(c), pe, row[i]) for sch, rows in t["E_phi"].items() if sch in schemes
            for c, row in rows.items() for i, pe in enumerate(t["Pe"])]


def sweep_entries(which: str):
    """Every printed DUGKS entry of the Zalesak ("zalesak") or smoothed-deformation
    ("deformation") tables: (table, scheme, cfl, Pe, M, E_phi)."""
    t = json.load(open(os.path.join(os.path.dirname(GOLDEN), f"{which}_e_phi.json")))
    out = []
    pt, mt = t["Pe_table"], t["M_table"]
    for sch, rows in pt["E_phi"].items():
        for c, row in rows.items():
            out += [("Pe", sch, float(c), pe, pt["M"], v) for pe, v in zip(pt["Pe"], row) if v is not None]
    for sch, rows in mt["E_phi"].items():
        for c, row in rows.items():
            out += [("M", sch, float(c), mt["Pe"], m, v) for m, v in zip(mt["M"], row) if v is not None]
    return out


def sweep_problem(which: str, scheme: str, cfl: float, Pe: float, M: float):
    order, flux, stages = SCHEMES[scheme]
    gen = WL.zalesak if which == "zalesak" else WL.deformation
    return dataclasses.replace(gen(Pe, cfl, M=M), order=order, flux=flux, stages=stages)


def step_function(phi: np.ndarray, phiA: float = 1.0, phiB: float = 0.0) -> np.ndarray:
    """Sec. III.B: at the final time phi is reset to phi_A or phi_B by its side of (phi_A + phi_B)/2."""
    return np.where(phi >= 0.5 * (phiA + phiB), phiA, phiB)
