"""Write the stored long-time Fourier evolutions used by the FP64 spectral parity test.

Each file holds U^t psi0 for one (lattice, box, mass, seed, t), evolved by
oracle.exact.evolve_mp (Sec. 4: DFT, D_k^t by repeated squaring in 50-digit
arithmetic, inverse DFT), in the device layout of include/qw.h, one complex value
per line ("re im", Python repr floats).  psi0 is inputs.random_field(dim, N, seed).
Calls only oracle/ and the seeded input generator.  Run from the repository root:

    python tests/golden/make_long_time_spectral.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import walk, exact  # noqa: E402
from paper_1603_06442_gb300 import inputs  # noqa: E402

CASES = [  # dim, N, m, seed, t
    (1, 64, 0.1, 3, 123457), (1, 64, 0.1, 3, 1000003), (1, 64, 0.1, 3, 10000019),
    (2, 8, 0.2, 4, 123457), (2, 8, 0.2, 4, 1000003), (2, 8, 0.2, 4, 10000019),
    (3, 8, 0.3, 5, 123457), (3, 8, 0.3, 5, 1000003),
]


def name(dim, N, m, seed, t):
    return "long_time_spectral_d%d_N%d_m%g_s%d_t%d.txt" % (dim, N, m, seed, t)


def main():
    for dim, N, m, seed, t in CASES:
        psi0 = walk.from_device(dim, N, inputs.random_field(dim, N, seed=seed))
        out = walk.to_device(dim, N, exact.evolve_mp(dim, m, psi0, t)).ravel()
        path = os.path.join(HERE, name(dim, N, m, seed, t))
        with open(path, "w") as f:
            f.write("# U^t psi0, dim=%d N=%d m=%r seed=%d t=%d; psi0 = inputs.random_field(dim, N, seed)\n"
                    % (dim, N, m, seed, t))
            f.write("# oracle.exact.evolve_mp (Sec. 4 Fourier form, D_k^t in 50 digits); device layout, re im\n")
            for v in out:
                f.write("%r %r\n" % (float(v.real), float(v.imag)))
        print(path)


if __name__ == "__main__":
    main()
