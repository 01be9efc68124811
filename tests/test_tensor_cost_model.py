"""Host model of the tensor-core cost kernel's arithmetic (csrc/cost_mma.cu), on the CPU.

The kernel computes the Hamming cost of Eq. (image_matching) for 62-bit census descriptors as
|a| + |b| - 2 a.b: A rows (-2 a_k, 1, 1), B rows (b_k, h, l) in e4m3, an fp32 accumulator per
(left pixel, right pixel) pair, then per lane a bias, a byte pack, a shift by the lane's band
offset and a byte reversal. This model follows the kernel's tile shape (128 left x 256 right
pixels), its epilogue warps (two per lane quarter), word and funnel shifts and the 255 rule, and
checks every cost word against the popcount of the XOR. It pins the index arithmetic and the
exactness of the encoding; the GPU parity tests check the kernel itself.
"""
import struct

import numpy as np

M, N, K = 128, 256, 64
EPQ = 2  # epilogue warps per lane quarter


def e4m3_small_int(v):
    if v == 0:
        return 0
    e = v.bit_length() - 1
    m = ((v << 3) >> e) & 7
    return ((e + 7) << 3) | m


def e4m3_value(b):
    s = -1.0 if b & 0x80 else 1.0
    e, m = (b >> 3) & 15, b & 7
    return s * (m / 8 * 2.0 ** -6 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7))


def test_operand_values_are_exact_in_e4m3():
    assert e4m3_value(0x38) == 1.0 and e4m3_value(0xC0) == -2.0
    for v in list(range(8)) + list(range(8, 57, 8)):
        assert e4m3_value(e4m3_small_int(v)) == v
    # every |b| of a 62-bit descriptor splits into h + l, both exact
    for nb in range(63):
        assert e4m3_value(e4m3_small_int(nb & 56)) + e4m3_value(e4m3_small_int(nb & 7)) == nb


def _bits(d):
    return [(int(d) >> k) & 1 for k in range(62)]


def _costs_model(ctl, ctr, D):
    W = len(ctl)
    out = np.zeros((W, D), np.uint8)
    DH = D // min(EPQ, D // 32)
    NP, NQ = (DH + 32) // 4, DH // 4
    for x0 in range(0, W, 128):
        A = np.zeros((M, K), np.float32)
        B = np.zeros((N, K), np.float32)
        for r in range(M):
            if x0 + r < W:
                A[r, :62] = [-2.0 * b for b in _bits(ctl[x0 + r])]
            A[r, 62:] = 1.0  # also rows past the image: their entries are not stored
        for j in range(N):
            xs = x0 - M + j
            if 0 <= xs < W:
                nb = bin(int(ctr[xs])).count("1")
                B[j, :62] = _bits(ctr[xs])
                B[j, 62] = e4m3_value(e4m3_small_int(nb & 56))
                B[j, 63] = e4m3_value(e4m3_small_int(nb & 7))
        acc = (A.astype(np.float64) @ B.T.astype(np.float64)).astype(np.float32)
        assert np.array_equal(acc, A.astype(np.float64) @ B.T.astype(np.float64))  # exact
        for warp in range(4 * (D // DH)):
            q, h = warp & 3, warp >> 2
            dh0 = h * DH
            ca = 32 * q + M - dh0 - DH
            assert ca % 32 == 0 and 0 <= ca and ca + 4 * NP <= N
            for lane in range(32):
                ti = 32 * q + lane
                x = x0 + ti
                la = bin(int(ctl[min(x, W - 1)])).count("1")
                bias = np.float32(la + 8388608.0)
                row = []
                for m in range(NP):  # packed low bytes of 4 columns
                    bts = [struct.unpack("<I", struct.pack("<f", np.float32(
                        acc[ti, ca + 4 * m + t] + bias)))[0] & 0xFF for t in range(4)]
                    row.append(bts[0] | bts[1] << 8 | bts[2] << 16 | bts[3] << 24)
                row.append(0)
                sh = lane + 1
                bs, ws = 8 * (sh & 3), sh >> 2
                o = [0] * NQ
                for n in range(NQ - 1, -1, -1):
                    w = ((row[ws + n + 1] << 32 | row[ws + n]) >> bs) & 0xFFFFFFFF
                    o[NQ - 1 - n] = int.from_bytes(w.to_bytes(4, "little")[::-1], "little")
                if x < dh0 + DH - 1:
                    for k in range(NQ):
                        nv = x - dh0 - 4 * k + 1
                        if nv <= 0:
                            o[k] = 0xFFFFFFFF
                        elif nv < 4:
                            o[k] |= (0xFFFFFFFF << (8 * nv)) & 0xFFFFFFFF
                if x < W:
                    out[x, dh0:dh0 + DH] = np.frombuffer(
                        b"".join(v.to_bytes(4, "little") for v in o), np.uint8)
    return out


def test_epilogue_gives_the_hamming_cost():
    rng = np.random.default_rng(7)
    for W, D in ((300, 128), (130, 64), (5, 128)):
        ctl = rng.integers(0, 2 ** 62, W, dtype=np.uint64)
        ctr = rng.integers(0, 2 ** 62, W, dtype=np.uint64)
        ctl[W // 2] = 0  # an all-zero descriptor inside the image (no bit set)
        got = _costs_model(ctl, ctr, D)
        want = np.array([[255 if x < d else bin(int(ctl[x]) ^ int(ctr[x - d])).count("1")
                          for d in range(D)] for x in range(W)], np.uint8)
        assert np.array_equal(got, want), (W, D, np.argwhere(got != want)[:3])
