"""CPU model of the tensor-core inverse FFT (csrc/fft_tc.cuh, csrc/tc_scale_block.cu).

The model replays the kernel's index arithmetic lane by lane in numpy: the
A/B/D fragment layouts of mma.sync.m16n8k16 (PTX ISA, "Matrix Fragments for
mma.m16n8k16"), the hi/lo split of both operands into FP16 or BF16, the
Stockham passes (pass 0 of radix 4 computed on the fly, radix 16 with
Ns = 4, 64 and 1024, the residue-class ownership of passes B and C), the XOR-swizzled
shared-memory layout, the sparse pass-0 inputs of a banded row, and the
cross-CTA radix-CL stage of a row split over CL residue classes.  Its result
must equal the inverse DFT of the row (numpy's FFT) to the split's precision,
and its shared-memory traffic must be a permutation (no slot written twice,
none read before written).  Tensor-core accumulation is modelled in FP64.
"""
import numpy as np
import pytest

NL, NB, Q0 = 16384, 1024, 4096


def tc_pad(i):
    i = np.asarray(i)
    lo = (0x23013210 >> (((i >> 6) & 7) * 4)) & 15
    hi = (0x9C14D850 >> (((i >> 10) & 7) * 4)) & 15
    return i ^ lo ^ hi


def round16(x, kind):
    x = np.asarray(x, np.float32)
    if kind == "f16":
        return x.astype(np.float16).astype(np.float32)
    # bf16: round to nearest even on the upper 16 bits of the float32
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split(v, kind):
    """v complex64 -> (hi, lo) complex with 16-bit parts (the kernel's tc_split)."""
    re, im = np.float32(v.real), np.float32(v.imag)
    hr, hi_ = round16(re, kind), round16(im, kind)
    lr, li = round16(re - hr, kind), round16(im - hi_, kind)
    return hr + 1j * hi_, lr + 1j * li


def afrag(kind):
    """The 32x32 real form of F16 (SIGN +1) assembled from each lane's fragments."""
    A = {"hi": np.zeros((32, 32)), "lo": np.zeros((32, 32))}
    for mt in range(2):
        for kt in range(2):
            for lane in range(32):
                g, t = lane >> 2, lane & 3
                for r in range(4):
                    q = g + 8 * (r & 1)
                    m = 8 * kt + t + 4 * (r >> 1)
                    e = (q * m) & 15
                    c, s = np.cos(2 * np.pi * e / 16), np.sin(2 * np.pi * e / 16)
                    a0, a1 = (c, -s) if mt == 0 else (s, c)
                    h, lo = split(np.complex64(a0 + 1j * a1), kind)
                    row = 16 * mt + g + 8 * (r & 1)         # fragment layout of A
                    col = 16 * kt + 2 * t + 8 * (r >> 1)
                    A["hi"][row, col], A["hi"][row, col + 1] = h.real, h.imag
                    A["lo"][row, col], A["lo"][row, col + 1] = lo.real, lo.imag
    return A


def mma_group(A, cols_hi, cols_lo):
    """cols_*[lane][h]: the B values lane (g, t) supplies for point m = t + 4h of
    column g.  Returns out[lane] = [(Re, Im) of output g, g+8 of columns 2t, 2t+1]."""
    B = {"hi": np.zeros((32, 8)), "lo": np.zeros((32, 8))}
    for name, cols in (("hi", cols_hi), ("lo", cols_lo)):
        for lane in range(32):
            g, t = lane >> 2, lane & 3
            for h in range(4):
                kt, reg = h >> 1, h & 1                  # fragment layout of B
                row = 16 * kt + 2 * t + 8 * reg
                B[name][row, g], B[name][row + 1, g] = cols[lane][h].real, cols[lane][h].imag
    D = A["hi"] @ B["lo"] + A["lo"] @ B["hi"] + A["hi"] @ B["hi"]
    out = []
    for lane in range(32):
        g, t = lane >> 2, lane & 3
        # fragment layout of D: rows g, g+8 of each m-tile at columns 2t, 2t+1
        y = {}
        for e in range(2):
            y[(g, 2 * t + e)] = D[g, 2 * t + e] + 1j * D[16 + g, 2 * t + e]
            y[(g + 8, 2 * t + e)] = D[8 + g, 2 * t + e] + 1j * D[24 + g, 2 * t + e]
        out.append(y)
    return out


def twiddle(k, m, Ns):
    return np.exp(2j * np.pi * k * m / (16 * Ns))


class Smem:
    def __init__(self):
        self.v = np.zeros(NL, np.complex128)
        self.written = np.zeros(NL, bool)

    def st(self, i, x):
        self.v[tc_pad(i)] = x
        self.written[tc_pad(i)] = True

    def ld(self, i):
        assert self.written[tc_pad(i)], "read before written"
        return self.v[tc_pad(i)]


def run_pass(sm, A, kind, Ns, groups, val, hold_check):
    """groups: list of (columns -> butterfly jj) per MMA; writes after all of a
    unit's reads (unit = one class for pass B, one MMA otherwise)."""
    for unit in groups:
        pending = []
        for jj_of in unit:
            cols_hi, cols_lo = [], []
            for lane in range(32):
                g, t = lane >> 2, lane & 3
                jj = jj_of(g)
                k = jj & (Ns - 1)
                hs, ls = [], []
                for h in range(4):
                    m = t + 4 * h
                    x = np.complex64(val(jj, m) * twiddle(k, m, Ns))
                    a, b = split(x, kind)
                    hs.append(a)
                    ls.append(b)
                cols_hi.append(hs)
                cols_lo.append(ls)
            pending.append((jj_of, mma_group(A, cols_hi, cols_lo)))
        for jj_of, out in pending:
            for lane in range(32):
                g, t = lane >> 2, lane & 3
                for e in range(2):
                    jj = jj_of(2 * t + e)
                    k = jj & (Ns - 1)
                    base = (jj - k) * 16 + k
                    for q in (g, g + 8):
                        hold_check.append(base + q * Ns)
                        sm.st(base + q * Ns, np.complex64(out[lane][(q, 2 * t + e)]))


def model_fft16384(x_local, kind, sparse_first=None):
    """The kernel's 16384-point FFT (SIGN +1) of one CTA's residue class."""
    A = afrag(kind)
    sm = Smem()

    def pass0_out(p):
        j, m0 = p >> 2, p & 3
        if sparse_first is not None:
            hit = sparse_first(j)
            if hit is None:
                return 0j
            r, x = hit
            return x * (1j ** ((r * m0) % 4))
        return sum(x_local[j + Q0 * r] * (1j ** ((r * m0) % 4)) for r in range(4))

    outs = []
    groups = [[(lambda n, jj0=(w + 16 * i) * 8: jj0 + n)] for w in range(16) for i in range(8)]
    run_pass(sm, A, kind, 4, groups, lambda jj, m: pass0_out(jj + NB * m), outs)
    assert sorted(outs) == list(range(NL))
    sm.written[:] = True
    for Ns, groups in (
        (64, [[(lambda n, k=4 * w + kk, rho=rho: k + 64 * (8 * rho + n)) for rho in range(2)]
              for w in range(16) for kk in range(4)]),
        # pass C on the same classes: butterflies k + 64 (8 rho + n)
        (1024, [[(lambda n, k=4 * w + kk, rho=rho: k + 64 * (8 * rho + n)) for rho in range(2)]
                for w in range(16) for kk in range(4)]),
    ):
        # every unit reads exactly the slots it writes (in-place closure)
        for unit in groups:
            reads = {jj_of(n) + NB * m for jj_of in unit for n in range(8) for m in range(16)}
            writes = set()
            for jj_of in unit:
                for n in range(8):
                    jj = jj_of(n)
                    k = jj & (Ns - 1)
                    writes |= {(jj - k) * 16 + k + q * Ns for q in range(16)}
            assert reads == writes
        outs = []
        snapshot = sm.v.copy()
        run_pass(sm, A, kind, Ns, groups, lambda jj, m, snap=snapshot: snap[tc_pad(jj + NB * m)], outs)
        assert sorted(outs) == list(range(NL))
    return np.array([sm.v[tc_pad(t)] for t in range(NL)])


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_tc_fft16384_dense_matches_inverse_dft(kind):
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(NL) + 1j * rng.standard_normal(NL)) * 2.0 ** -7  # L1 below 2^15
    X = model_fft16384(x, kind)
    ref = np.fft.ifft(x) * NL
    err = np.abs(X - ref).max() / np.abs(ref).max()
    assert err < (1e-5 if kind == "f16" else 2e-4), err


def test_tc_cluster_row_banded_matches_inverse_dft():
    """A banded 131072-point row on 8 residue classes: sparse pass 0 per class
    (the kernel's `first`), then the cross-CTA radix-8 stage, equals the
    inverse DFT of the row."""
    CL, N = 8, 8 * NL
    rng = np.random.default_rng(3)
    b0, B = 130000, 9000          # a band that wraps past N
    Y = np.zeros(N, np.complex128)
    idx = (b0 + np.arange(B)) % N
    Y[idx] = rng.standard_normal(B) + 1j * rng.standard_normal(B)
    Y *= 2.0 ** 15 / np.abs(Y).sum()
    A_c = []
    for rank in range(CL):
        delta = (rank - b0) & (CL - 1)
        Bm = (B - delta + CL - 1) // CL if delta < B else 0
        m_first = ((((b0 + delta) & (N - 1)) - rank) // CL) & (NL - 1)
        assert Bm <= Q0

        def first(j, rank=rank, Bm=Bm, m_first=m_first):
            d0 = (j - m_first) & (Q0 - 1)
            if d0 >= Bm:
                return None
            m = (m_first + d0) & (NL - 1)
            r = (m - j) // Q0
            assert 0 <= r < 4 and (m - j) % Q0 == 0
            return r, Y[rank + CL * m]

        A_c.append(model_fft16384(None, "f16", sparse_first=first))
    t1 = np.arange(NL)
    out = np.zeros(N, np.complex128)
    for q in range(CL):  # CTA q's t1 range
        tt = t1[q * (NL // CL):(q + 1) * (NL // CL)]
        v = np.stack([A_c[c][tt] * np.exp(2j * np.pi * c * tt / N) for c in range(CL)])
        for t2 in range(CL):
            out[tt + NL * t2] = sum(v[c] * np.exp(2j * np.pi * c * t2 / CL) for c in range(CL))
    ref = np.fft.ifft(Y) * N
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-5


def test_swizzle_is_a_permutation_and_conflict_free():
    """tc_pad permutes the 16384 slots; every warp access of the passes and
    the natural-order reads touches 16 distinct 8-byte bank pairs per
    half-warp."""
    assert np.array_equal(np.sort(tc_pad(np.arange(NL))), np.arange(NL))

    def ok(addrs):
        a = tc_pad(np.asarray(addrs))
        return all(len(set(a[h:h + 16] & 15)) == 16 for h in (0, 16))

    lanes = np.arange(32)
    g, t = lanes >> 2, lanes & 3
    for w in range(16):
        for i in range(8):
            jj0 = (w + 16 * i) * 8
            for e in range(2):
                jj = jj0 + 2 * t + e
                for qh in (0, 8):
                    k = jj & 3
                    assert ok((jj - k) * 16 + k + 4 * (g + qh))              # pass A stores
        for kk in range(4):
            k = 4 * w + kk
            for rho in range(2):
                for h in range(4):
                    assert ok(k + 64 * (8 * rho + g) + NB * (t + 4 * h))     # pass B, C loads
                for e in range(2):
                    for qh in (0, 8):
                        jj = k + 64 * (8 * rho + 2 * t + e)
                        assert ok((jj - k) * 16 + k + 64 * (g + qh))         # pass B stores
                        assert ok(jj + 1024 * (g + qh))                      # pass C stores
    for base in range(0, NL, 32):
        assert ok(base + lanes)                                              # natural order


def test_hoisted_swizzle_terms_equal_tc_pad():
    """Passes B and C XOR fixed per-lane terms instead of evaluating tc_pad on
    every access; those terms equal tc_pad's on every index they touch."""
    lut = lambda b: (0x9C14D850 >> (b * 4)) & 15  # noqa: E731
    lut_lo = lambda b: (0x23013210 >> (b * 4)) & 15  # noqa: E731
    lanes = np.arange(32)
    g, t = lanes >> 2, lanes & 3
    for w in range(16):
        for kk in range(4):
            k = 4 * w + kk
            for rho in range(2):
                for h in range(4):
                    i = k + 64 * (8 * rho + g) + NB * (t + 4 * h)
                    assert np.array_equal(i ^ (lut_v(lut_lo, g) ^ lut_v(lut, (t + 4 * h) & 7)), tc_pad(i))
                for e in range(2):
                    for qh in (0, 8):
                        i = 1024 * (8 * rho + 2 * t + e) + k + 64 * (g + qh)
                        assert np.array_equal(i ^ (lut_v(lut_lo, g) ^ lut_v(lut, 2 * t + e)), tc_pad(i))
                        i = k + 64 * (8 * rho + 2 * t + e) + 1024 * (g + qh)
                        assert np.array_equal(i ^ (lut_v(lut_lo, 2 * t + e) ^ lut_v(lut, g)), tc_pad(i))


def lut_v(lut, b):
    return np.vectorize(lut)(np.asarray(b))
