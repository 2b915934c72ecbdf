"""Counter-based Philox generator for the oracle (test infrastructure only).

The paper draws one uniform variate xi in [0,1) per sampling decision (Section 2.2,
"Sampling Techniques").  It does not fix a generator; the lookup library keys a
counter-based generator on (query, sample) so that every query's variates are a
pure function of its index.  The generator is Philox from Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written here from
its published definition:

* state: a counter of four W-bit words and a key of two W-bit words;
* one round: the products M0*c0 and M1*c2 are split into high and low W-bit
  halves, and the new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
* between rounds the key is bumped by the Weyl constants (W0, W1);
* ten rounds.

The round structure below is written once for any word width.  Its 64-bit
instantiation is checked against numpy's independent ``Philox`` bit generator
(which is Philox4x64-10), which pins the structure; the lookup library uses the
32-bit instantiation with the published 4x32 multipliers and Weyl constants.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may use anything in ``oracle/``.
"""
import numpy as np

# Published Philox constants (Salmon et al., SC'11, Table 2 and Section 4.2).
PHILOX4X32 = {"bits": 32, "M": (0xD2511F53, 0xCD9E8D57), "W": (0x9E3779B9, 0xBB67AE85)}
PHILOX4X64 = {"bits": 64, "M": (0xD2E7470EE14C6C93, 0xCA5A826395121157),
              "W": (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)}

ROUNDS = 10


def _mulhilo32(m, c):
    # c is a uint64 array holding 32-bit words; m < 2^32 so the product fits 64 bits.
    p = np.uint64(m) * c
    return p >> np.uint64(32), p & np.uint64(0xFFFFFFFF)


def _mulhilo64(m, c):
    # Python integers: exact 128-bit product.
    p = m * c
    return p >> 64, p & ((1 << 64) - 1)


def philox4(ctr, key, spec, rounds=ROUNDS):
    """Philox4xW-R on a counter (c0, c1, c2, c3) and key (k0, k1).

    Words are numpy uint64 arrays (W = 32) or Python ints (W = 64).  Returns the
    four output words.
    """
    bits = spec["bits"]
    mask = (1 << bits) - 1
    m0, m1 = spec["M"]
    w0, w1 = spec["W"]
    mulhilo = _mulhilo32 if bits == 32 else _mulhilo64
    c0, c1, c2, c3 = ctr
    k0, k1 = key
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + w0) & mask
            k1 = (k1 + w1) & mask
        hi0, lo0 = mulhilo(m0, c0)
        hi1, lo1 = mulhilo(m1, c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox4x32(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Counter words may be arrays; returns four uint64
    arrays holding 32-bit outputs."""
    u = lambda a: np.asarray(a, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    c = np.broadcast_arrays(u(c0), u(c1), u(c2), u(c3))
    return philox4(tuple(c), (int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF), PHILOX4X32)


def philox4x64(ctr, key):
    """Scalar Philox4x64-10 on Python ints (used only to pin the round structure)."""
    return philox4(tuple(int(x) for x in ctr), tuple(int(x) for x in key), PHILOX4X64)


def query_variates(qid, sample_index, seed, stream=0):
    """The four uniform variates of one lookup, shape (4, N), float64.

    Counter = (qid low word, qid high word, sample index, stream); key = (seed low
    word, seed high word).  Stream 0 serves every filter; the positivized filter also
    draws stream 1.  Each 32-bit output keeps its top 24 bits:
    u = (r >> 8) * 2^-24, which is exact in both float32 and float64 and lies in
    [0, 1).  Word 0 drives the x axis, 1 the y axis, 2 the z axis and 3 the MIP
    level choice.
    """
    q = np.asarray(qid, dtype=np.uint64)
    seed = int(seed) & ((1 << 64) - 1)
    r = philox4x32(q & np.uint64(0xFFFFFFFF), q >> np.uint64(32),
                   np.uint64(int(sample_index) & 0xFFFFFFFF), np.uint64(int(stream) & 0xFFFFFFFF),
                   seed & 0xFFFFFFFF, seed >> 32)
    return np.stack([(w >> np.uint64(8)).astype(np.float64) * 2.0 ** -24 for w in r])
