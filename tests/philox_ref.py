"""Philox4x32-10 written out from its published definition (Salmon et al.,
SC'11): ten rounds of two 32x32->64-bit multiplies by 0xD2511F53 and
0xCD9E8D57 with the xor/permute network, key bumped by the Weyl constants
0x9E3779B9 and 0xBB67AE85 between rounds.  Used to check the GPU generator
bit for bit."""
from pathlib import Path

M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    m0, m1 = 0xD2511F53, 0xCD9E8D57
    w0, w1 = 0x9E3779B9, 0xBB67AE85
    c0, c1, c2, c3 = (int(v) & M32 for v in ctr)
    k0, k1 = (int(v) & M32 for v in key)
    for _ in range(10):
        p0 = m0 * c0
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & M32, p1 & M32, ((p0 >> 32) ^ c3 ^ k1) & M32, p0 & M32
        k0 = (k0 + w0) & M32
        k1 = (k1 + w1) & M32
    return c0, c1, c2, c3


def load_kat():
    path = Path(__file__).parent / "golden" / "philox4x32_10_kat.txt"
    out = []
    for line in path.read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        out.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return out
