"""Write ``saturation_64x24x32.json``: the FP64 CPU oracle run to saturation.

Runs the oracle (its OpenMP build, bitwise equal to the serial one) on the
``saturation_64x24x32`` workload of ``synth.WORKLOADS`` for each applied
field of its sweep, from f = 0 and sigma = 0, until the convergence test of
Sec. 2 (Sun et al., arXiv 2303.14119: sigma and both wall fluxes change by
less than the tolerance over the window) passes, and stores the saturated
step and the history row there.  Calls nothing but ``oracle/``; the CUDA
library never writes these values.

    python tests/golden/make_saturation.py
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2303_14119_gb300 import synth  # noqa: E402

NAME = "saturation_64x24x32"
OUT = os.path.join(HERE, NAME + ".json")
CHUNK = 5000


def run_to_saturation(Ey, threads=0):
    """One oracle run of the workload at field Ey until it saturates (or the
    workload's step cap): returns the oracle, its saturated step and the
    history up to the last step taken."""
    w = synth.WORKLOADS[NAME]
    o = oracle.Oracle(w["nx"], w["nv1"], w["nv2"], w["h_max"], -w["v1_span"], w["v1_span"],
                      -w["v2_span"], w["v2_span"], cfl=w["cfl"], threads=threads or os.cpu_count())
    o.set_fields(Ey)
    o.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
    o.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
    o.set_convergence(w["sat_window"], w["sat_tol"])
    while o.info()["step"] < w["steps"] and o.info()["sat_step"] < 0:
        o.step(CHUNK)
    return o, o.info()["sat_step"], o.history()


def record(Ey):
    w = synth.WORKLOADS[NAME]
    o, sat, hist = run_to_saturation(Ey)
    row = hist[sat]
    A1 = oracle.first_crossover(w["delta_max"], w["A_max"], w["k_s"])
    return {
        "Ey": Ey, "sat_step": int(sat), "dt": o.info()["dt"],
        "sigma_sat": float(row[2]), "gamma_pe_sat": float(row[3]), "gamma_see_sat": float(row[4]),
        "N_sat": float(row[6]), "Ex0_sat": float(row[7]),
        "sigma_every_5000": [float(hist[s][2]) for s in range(5000, sat + 1, 5000)],
        "A1_eV": A1, "sigma_eq20": oracle.sigma_eq20(Ey, w["T_se"], A1),
    }


def main():
    w = synth.WORKLOADS[NAME]
    out = {"_source": "FP64 CPU oracle (oracle/fk_oracle.c) on synth.WORKLOADS['%s'], written by "
                      "tests/golden/make_saturation.py; convergence test of Sec. 2" % NAME,
           "window": w["sat_window"], "tol": w["sat_tol"],
           "runs": [record(Ey) for Ey in w["Ey_sweep"]]}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out["runs"], indent=1))


if __name__ == "__main__":
    main()
