"""Writes c1_tracer_1000.txt: the oracle's square-basin tracer run (32x32 squares
split in two, 10 sigma layers, solid-body rotation, Gaussian blob, dt = 5 s,
kappa_v = 1e-3) after 0 and 1000 steps of the explicit-horizontal / implicit-
vertical SSP-RK3 scheme (Sec. 2.3, Eqs. 11-14).  Calls only oracle/ and the seeded
input generators.  Run: python tests/golden/make_c1_tracer_1000.py  (about 25 min)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import tracer as otr  # noqa: E402
from oracle.mesh import OMesh  # noqa: E402

STEPS = 1000
N_SAMPLES = 256


def main():
    W = wl.WORKLOADS["square_tracer"]
    m = W["mesh"]()
    u, v = wl.c1_velocity(m)
    T = wl.c1_tracer(m)
    om = OMesh(m)
    eta = np.zeros((3, m.n_tri))
    Tn = otr.to3(T, om.P)
    uu, vv = otr.to3(u, om.P), otr.to3(v, om.P)
    m0 = otr.tracer_mass(om, eta, Tn)
    for n in range(STEPS):
        eta, Tn, _ = otr.tracer_step(om, eta, Tn, uu, vv, W["dt"], W["kappa_v"])
    m1 = otr.tracer_mass(om, eta, Tn)
    flat = Tn.ravel()
    idx = np.sort(np.random.default_rng(2605).choice(flat.size, N_SAMPLES, replace=False))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_tracer_1000.txt")
    with open(out, "w") as fh:
        fh.write("# Oracle (FP64, CPU) square-basin tracer run after %d steps, written by\n" % STEPS)
        fh.write("# tests/golden/make_c1_tracer_1000.py: config of the explicit-horizontal /\n")
        fh.write("# implicit-vertical tracer scheme (Sec. 2.3, Eqs. 11-14), square 10 km basin,\n")
        fh.write("# 2048 triangles x 10 layers, dt = 5 s, kappa_v = 1e-3.\n")
        fh.write("# node index = (c*3 + a) * P + prism (the library's field layout)\n")
        fh.write(f"steps {STEPS}\n")
        fh.write(f"mass0 {m0!r}\n")
        fh.write(f"mass {m1!r}\n")
        fh.write(f"l2 {float(np.sqrt(np.sum(flat ** 2)))!r}\n")
        for i in idx:
            fh.write(f"{int(i)} {float(flat[i])!r}\n")
    print(out)


if __name__ == "__main__":
    main()
