"""Writes channel128_member5_2steps.txt: sampled values of one member of the
128 x 97 x 128 constant-flux Poiseuille ensemble (Re = 3250, Re_tau ~ 180,
box 4 pi x 2 x 4 pi / 3, dt = 0.002; seeded state of 16 members with a
k^-5/3 spectrum at 10 % amplitude) after two steps of the oracle.

Calls only the oracle and the seeded input generator.  Run from the repository
root:  python tests/golden/make_channel128_samples.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import dns_synth  # noqa: E402
import oracle  # noqa: E402

MX, MY, MZ = 128, 97, 128
LX, LZ, RE, DT = 4 * np.pi, 4 * np.pi / 3, 3250.0, 0.002
MEMBERS, SEED0, AMP, MEMBER, STEPS = 16, 5000, 1e-1, 5, 2
NSAMPLE = 400


def main():
    st = dns_synth.make_state(MX, MY, MZ, LX, LZ, "poiseuille", MEMBERS, SEED0, AMP, spectrum="kolmogorov")
    x = tuple(st[k][MEMBER:MEMBER + 1] for k in ("v", "eta", "U", "W"))
    ch = oracle.Channel(MX, MY, MZ, LX, LZ, RE, DT, "poiseuille")
    v, eta, U, W = ch.step(x, STEPS)
    ny, nkz, nkx = v.shape[1:]
    rng = np.random.default_rng(128)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "channel128_member5_2steps.txt")
    with open(out, "w") as f:
        f.write("# Oracle (oracle.Channel, FP64) after %d steps of member %d of the seeded\n" % (STEPS, MEMBER))
        f.write("# dns_synth.make_state(%d, %d, %d, 4pi, 4pi/3, 'poiseuille', %d, %d, %g, spectrum='kolmogorov'),\n"
                % (MX, MY, MZ, MEMBERS, SEED0, AMP))
        f.write("# Re = %g, dt = %g.  Written by tests/golden/make_channel128_samples.py.\n" % (RE, DT))
        f.write("# max |v|, max |eta| over the member's whole state:\n")
        f.write("scale %.17e %.17e\n" % (np.abs(v).max(), np.abs(eta).max()))
        f.write("# field y_interior m_index n re im  (m_index = m + Kz)\n")
        for name, a in (("v", v), ("eta", eta)):
            ys = rng.integers(0, ny, NSAMPLE)
            ms = rng.integers(0, nkz, NSAMPLE)
            ns = rng.integers(0, nkx, NSAMPLE)
            for y, m, n in zip(ys, ms, ns):
                c = a[0, y, m, n]
                f.write("%s %d %d %d %.17e %.17e\n" % (name, y, m, n, c.real, c.imag))
        f.write("# profiles: U j value, W j value (all My nodes)\n")
        for name, a in (("U", U), ("W", W)):
            for j in range(MY):
                f.write("%s %d %.17e\n" % (name, j, a[0, j]))
    print("wrote", out)


if __name__ == "__main__":
    main()
