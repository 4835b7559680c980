"""Writes cavity64_re100_t2000.txt, the oracle's own 64 x 64 lid-driven cavity after 2000 updates.

This is a regression fixture of the oracle: it calls nothing but `oracle/`.  The case is a cavity
with three halfway bounce-back walls and a lid moving at U = 0.1 (moving-wall bounce-back,
rho_w = 1).  Re = U L / nu = 100 with L = 64 gives tau = 3 nu + 1/2 = 0.692.  The run starts
from rest, f = w (Eq. feq-full with rho = 1, u = 0), and applies the SmrtLBM update
(Eq. SmrtLBM-1) 2000 times.

Stored (17 significant digits):
- u_x on the column i = 32 and u_y on the row j = 32;
- rho at four nodes and the total mass;
- two weighted checksums of the whole population field, sum f * (1 + a + j/64 + i/4096) and
  sum f * (-1)^(a+i+j), which react to any change anywhere in the field.
The header carries the SHA-256 of oracle/smrt_oracle.c and the commit that last changed it.

Run from the repository root:  python tests/golden/make_cavity64.py
"""
import hashlib
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

N, U, RE, STEPS = 64, 0.1, 100.0, 2000
TAU = 3.0 * U * N / RE + 0.5
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity64_re100_t2000.txt")


def fields():
    f = O.run(O.cavity_initial(N, N), STEPS, O.CAVITY, TAU, u_lid=U)
    rho, u = O.macros(f)
    a, j, i = np.meshgrid(np.arange(9), np.arange(N), np.arange(N), indexing="ij")
    return {
        "ux_column_i32": u[0][:, 32],
        "uy_row_j32": u[1][32, :],
        "rho_nodes_j_i": np.array([rho[0, 0], rho[N - 1, 0], rho[32, 32], rho[N - 1, N - 1]]),
        "mass": np.array([rho.sum()]),
        "checksum_weighted": np.array([(f * (1.0 + a + j / 64.0 + i / 4096.0)).sum()]),
        "checksum_alternating": np.array([(f * (-1.0) ** (a + i + j)).sum()]),
    }


def read(path=OUT):
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, vals = line.split(":", 1)
            out[key.strip()] = np.array([float(v) for v in vals.split()])
    return out


def main():
    src = os.path.join(ROOT, "oracle", "smrt_oracle.c")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    try:
        commit = subprocess.run(["git", "log", "-1", "--format=%H", "--", "oracle/smrt_oracle.c"], cwd=ROOT,
                                capture_output=True, text=True, check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        commit = "unknown"
    with open(OUT, "w") as fh:
        fh.write("# 64 x 64 lid-driven cavity, U_lid = 0.1, Re = 100, tau = %.17g, %d SmrtLBM updates from rest\n"
                 % (TAU, STEPS))
        fh.write("# (Eq. SmrtLBM-1 with halfway and moving-wall bounce-back; written by tests/golden/make_cavity64.py)\n")
        fh.write("# oracle/smrt_oracle.c sha256 %s, last changed in commit %s\n" % (sha, commit))
        for key, vals in fields().items():
            fh.write("%s: %s\n" % (key, " ".join("%.17g" % v for v in vals)))
    print(OUT)


if __name__ == "__main__":
    main()
