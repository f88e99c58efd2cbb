"""Host-side model of the mixed-radix row (no GPU): the Stockham passes, with
the indexing the smooth-length kernels use, run in numpy under the schedules
the library's scheduler picks (cwt_smooth_schedule), must reproduce the DFT;
the magic divisors must give exact quotients for every butterfly; and the
padded shared-memory index must satisfy the identities that the fixed-length
kernels' linear addressing relies on.

The pass structure (Section "Fast Fourier transform": 2,3,5,7-smooth lengths):
pass p has radix R and Ns = R_0 ... R_{p-1}; butterfly b < N/R takes the
inputs b + r N/R, multiplies input r by w^r with w = exp(SIGN 2 pi i k / (Ns R))
and k = b mod Ns, runs an R-point DFT and writes output r to
(b - k) R + k + r Ns.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p


LENGTHS = [35, 98, 250, 500, 1000, 1215, 2000, 2401, 2500, 3024, 4000, 5000, 6000, 7500, 8000,
           10000, 12000, 14000]


def stockham(x, radices, sign):
    """The kernels' pass sequence on one row (complex128)."""
    N = len(x)
    cur = np.asarray(x, dtype=np.complex128).copy()
    Ns = 1
    for R in radices:
        nb = N // R
        b = np.arange(nb)
        k = b % Ns
        v = np.stack([cur[b + r * nb] for r in range(R)])              # [R][nb]
        w = np.exp(sign * 2j * np.pi * k / (Ns * R))
        v = v * w[None, :] ** np.arange(R)[:, None]                   # twiddles w^r
        F = np.exp(sign * 2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
        y = F @ v                                                     # R-point DFT
        out = np.empty_like(cur)
        for r in range(R):
            out[(b - k) * R + k + r * Ns] = y[r]
        cur = out
        Ns *= R
    return cur


@pytest.mark.parametrize("N", LENGTHS)
def test_scheduled_passes_compute_the_dft(lib, N):
    radices, T, pair, fixed = lib.cwt_smooth_schedule(N)
    assert int(np.prod(radices)) == N
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    # forward (SIGN = -1) and inverse (SIGN = +1, unnormalised; the bank carries 1/N)
    np.testing.assert_allclose(stockham(x, radices, -1), np.fft.fft(x), rtol=0, atol=1e-9 * N)
    np.testing.assert_allclose(stockham(x, radices, +1), np.fft.ifft(x) * N, rtol=0, atol=1e-9 * N)


def magic(d):
    """ceil(2^32 / d), 0 for d = 1: the divisor constant of the kernels."""
    return 0 if d <= 1 else ((1 << 32) + d - 1) // d


@pytest.mark.parametrize("N", LENGTHS)
def test_magic_divisors_are_exact(lib, N):
    """q = umulhi(b, ceil(2^32 / Ns)) equals b // Ns for every butterfly b of
    every pass (b < N/R < 2^14, Ns <= 2^13: division by invariant integers),
    and the narrow-band first pass's divisions by N/R_0 of values below 2N."""
    radices, _, _, _ = lib.cwt_smooth_schedule(N)
    Ns = 1
    for R in radices:
        nb = N // R
        b = np.arange(nb, dtype=np.uint64)
        if Ns > 1:
            q = (b * np.uint64(magic(Ns))) >> np.uint64(32)
            np.testing.assert_array_equal(q, b // np.uint64(Ns))
        Ns *= R
    # first pass, narrow band: b - b0 + N (mod nb) and (e - b) / nb, both below 2N
    nb0 = N // radices[0]
    d = np.arange(0, 2 * N, dtype=np.uint64)
    q = (d * np.uint64(magic(nb0))) >> np.uint64(32)
    np.testing.assert_array_equal(q, d // np.uint64(nb0))


def spad2(i):
    return i + (i >> 4)


def test_padded_index_identities():
    """spad2(i) = i + i/16 (one pad slot every 16 float2).  A run of accesses
    with a stride that is a multiple of 16 is one padded base plus constant
    offsets, spad2(x + 16 m) = spad2(x) + 17 m; a first-pass butterfly of a
    radix that is a multiple of 16 writes spad2(b R) + spad2(r)."""
    x = np.arange(0, 20000)
    for m in (1, 2, 25, 400, 625):
        np.testing.assert_array_equal(spad2(x + 16 * m), spad2(x) + 17 * m)
    b = np.arange(0, 700)
    for R in (16, 32):
        for r in range(R):
            np.testing.assert_array_equal(spad2(b * R + r), spad2(b * R) + spad2(r))
    # the strides of the 10000-point fixed kernel (16 x 25 x 25) are all multiples of 16
    N, Ns = 10000, 1
    for R in (16, 25, 25):
        if Ns > 1:
            assert (N // R) % 16 == 0 and Ns % 16 == 0
        Ns *= R


def pow2_radices(N, R):
    """Pass radices of a power-of-two row with R points per thread: the
    leftover factor 2^(log2 N mod log2 R) first (or R), then R per pass."""
    L, r = N.bit_length() - 1, R.bit_length() - 1
    R0 = 1 << (L % r) if L % r else R
    return [R0] + [R] * ((L - (R0.bit_length() - 1)) // r)


@pytest.mark.parametrize("N,R", [(32, 16), (512, 16), (2048, 16), (8192, 16), (8192, 32),
                                 (16384, 32)])
def test_power_of_two_passes_compute_the_dft(N, R):
    radices = pow2_radices(N, R)
    assert int(np.prod(radices)) == N and all(q <= R for q in radices)
    rng = np.random.default_rng(N + R)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    np.testing.assert_allclose(stockham(x, radices, -1), np.fft.fft(x), rtol=0, atol=1e-9 * N)
    np.testing.assert_allclose(stockham(x, radices, +1), np.fft.ifft(x) * N, rtol=0, atol=1e-9 * N)


@pytest.mark.parametrize("N,f", [(64, 2), (1024, 4), (4096, 8), (16384, 16)])
def test_spectral_fold_gives_every_fth_sample(N, f):
    """Decimation by a power-of-two factor f: the N/f-point inverse DFT of the
    folded spectrum Y'[j] = sum_q Y[j + q N/f] is exactly every f-th sample of
    the N-point inverse DFT (up to the 1/N vs f/N scaling)."""
    rng = np.random.default_rng(N * f)
    Y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    M = N // f
    folded = Y.reshape(f, M).sum(axis=0)
    np.testing.assert_allclose(np.fft.ifft(folded) / f, np.fft.ifft(Y)[::f], rtol=0, atol=1e-12)


def test_narrow_band_first_pass_position():
    """Pass 0 with a band [b0, b0 + B) (mod N) no wider than nb = N/R_0: the
    inputs b + r nb of butterfly b meet the band at most once, at
    e = b0 + ((b - b0) mod nb) (mod N) when (b - b0) mod nb < B, in position
    r = (e - b) / nb -- brute force over every butterfly."""
    rng = np.random.default_rng(7)
    for N, R0 in ((10000, 16), (5000, 8), (2000, 10), (16384, 16), (500, 20)):
        nb = N // R0
        for _ in range(20):
            b0 = int(rng.integers(0, N))
            B = int(rng.integers(1, nb + 1))
            band = set(((b0 + np.arange(B)) % N).tolist())
            for b in range(nb):
                hits = [r for r in range(R0) if b + r * nb in band]
                u = (b - b0) % nb
                if u < B:
                    e = (b0 + u) % N
                    assert e % nb == b % nb and e >= b
                    assert hits == [(e - b) // nb]
                else:
                    assert hits == []


@pytest.mark.parametrize("CL,NL", [(2, 64), (4, 256), (8, 512), (8, 16384)])
def test_cluster_decomposition(CL, NL):
    """Rows of N = CL NL points on a cluster of CL CTAs: with k = c + CL m and
    t = t1 + NL t2, X[t1 + NL t2] = sum_c w_CL^(c t2) w_N^(c t1) A_c[t1], A_c
    the NL-point DFT of residue class c; CTA c emits t1 in [c NL/CL,
    (c+1) NL/CL) for every t2, so the CTAs' outputs cover the row once."""
    N = CL * NL
    rng = np.random.default_rng(CL * NL)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    for sign, ref in ((-1, np.fft.fft(x)), (+1, np.fft.ifft(x) * N)):
        A = np.stack([stockham(x[c::CL], pow2_radices(NL, 32 if NL >= 32 else NL), sign)
                      for c in range(CL)])                                # [CL][NL]
        t1 = np.arange(NL)
        X = np.empty(N, dtype=np.complex128)
        owner = np.full(N, -1)
        for cta in range(CL):
            span = slice(cta * NL // CL, (cta + 1) * NL // CL)
            for t2 in range(CL):
                acc = sum(np.exp(sign * 2j * np.pi * c * t2 / CL)
                          * np.exp(sign * 2j * np.pi * c * t1[span] / N) * A[c, span] for c in range(CL))
                X[t1[span] + NL * t2] = acc
                assert (owner[t1[span] + NL * t2] == -1).all()
                owner[t1[span] + NL * t2] = cta
        assert (owner >= 0).all()
        np.testing.assert_allclose(X, ref, rtol=0, atol=1e-9 * N)


def _factor_split(R):
    """The kernels' first factor of a composite radix: its power-of-two part,
    else its smallest prime."""
    if R % 2 == 0:
        return R & -R
    return 3 if R % 3 == 0 else 5 if R % 5 == 0 else 7


@pytest.mark.parametrize("R", [6, 10, 12, 14, 15, 18, 20, 21, 24, 28, 30])
def test_prime_factor_maps(R):
    """Composite radices whose two factors are coprime run the prime-factor
    (Good-Thomas) algorithm without inner twiddles: inputs gathered at
    (R2 n1 + R1 n2) mod R, an R1-point DFT over n1, an R2-point DFT over n2,
    output (k1, k2) stored at (k1 R2 u2 + k2 R1 u1) mod R with u2 = R2^-1
    mod R1 and u1 = R1^-1 mod R2 -- the maps must give the R-point DFT."""
    R1 = _factor_split(R)
    R2 = R // R1
    assert np.gcd(R1, R2) == 1
    u2, u1 = pow(R2, -1, R1), pow(R1, -1, R2)
    rng = np.random.default_rng(R)
    x = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    for sign in (-1, +1):
        F1 = np.exp(sign * 2j * np.pi * np.outer(np.arange(R1), np.arange(R1)) / R1)
        F2 = np.exp(sign * 2j * np.pi * np.outer(np.arange(R2), np.arange(R2)) / R2)
        g = np.array([[x[(R2 * n1 + R1 * n2) % R] for n1 in range(R1)] for n2 in range(R2)])  # [n2][n1]
        t = g @ F1.T                     # [n2][k1]
        y = F2 @ t                       # [k2][k1]
        X = np.empty(R, dtype=np.complex128)
        for k1 in range(R1):
            for k2 in range(R2):
                X[(k1 * R2 * u2 + k2 * R1 * u1) % R] = y[k2, k1]
        ref = np.exp(sign * 2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R) @ x
        np.testing.assert_allclose(X, ref, rtol=0, atol=1e-12 * R)


@pytest.mark.parametrize("CL,NL", [(3, 4725), (2, 7203), (5, 3125), (6, 2560), (7, 2240), (8, 15360),
                                   (9, 1000), (10, 12288), (12, 2500), (16, 7680)])
def test_smooth_cluster_decomposition(lib, CL, NL):
    """Smooth rows on clusters (any CL in 2 ... 16): the residue classes run the
    scheduler's NL-point passes, the cross-CTA radix-CL stage finishes the row;
    the class's in-band bins are the cyclic run of Bm local points from
    m_first (delta = (c - b0) mod CL, Bm = ceil((B - delta) / CL)), and with
    Bm <= NL / R_0 each first-pass butterfly meets at most one of them."""
    N = CL * NL
    radices = lib.cwt_smooth_schedule(NL)[0]
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    for sign, ref in ((-1, np.fft.fft(x)), (+1, np.fft.ifft(x) * N)):
        A = np.stack([stockham(x[c::CL], radices, sign) for c in range(CL)])
        t1 = np.arange(NL)
        X = np.empty(N, dtype=np.complex128)
        for cta in range(CL):
            span = slice(cta * NL // CL, (cta + 1) * NL // CL)
            for t2 in range(CL):
                X[t1[span] + NL * t2] = sum(np.exp(sign * 2j * np.pi * c * t2 / CL)
                                            * np.exp(sign * 2j * np.pi * c * t1[span] / N) * A[c, span]
                                            for c in range(CL))
        np.testing.assert_allclose(X, ref, rtol=0, atol=1e-9 * N)
    nb = NL // radices[0]
    for _ in range(30):
        b0 = int(rng.integers(0, N))
        B = int(rng.integers(1, N // 4))
        band = np.zeros(N, dtype=bool)
        band[(b0 + np.arange(B)) % N] = True
        for c in range(CL):
            delta = (c - b0) % CL
            Bm = -(-(B - delta) // CL) if delta < B else 0
            m_first = ((((b0 + delta) % N) - c) // CL) % NL
            run = (m_first + np.arange(Bm)) % NL
            assert sorted(run.tolist()) == np.flatnonzero(band[c::CL]).tolist()
            if Bm <= nb:
                for b in range(nb):
                    hits = [r for r in range(radices[0]) if band[c + CL * (b + r * nb)]]
                    u = (b - m_first) % nb
                    if u < Bm:
                        m = (m_first + u) % NL
                        assert hits == [(m - b) // nb]
                    else:
                        assert hits == []


def _half_warp_degree(addrs):
    """Most distinct float2 addresses one of 16 eight-byte bank pairs serves in
    one half-warp of 64-bit shared-memory accesses (1: no bank conflict)."""
    worst = 1
    for h in range(0, len(addrs), 16):
        banks = {}
        for a in addrs[h:h + 16]:
            if a is not None:
                banks.setdefault(a & 15, set()).add(a)
        if banks:
            worst = max(worst, max(len(s) for s in banks.values()))
    return worst


@pytest.mark.parametrize("N,T,radices", [(10000, 416, (16, 25, 25)), (8000, 416, (16, 25, 20)),
                                          (12000, 512, (16, 25, 30)), (15360, 512, (16, 30, 32)),
                                          (14400, 512, (16, 30, 30))])
def test_fixed_pass_addressing_is_bank_conflict_free(N, T, radices):
    """The staging addresses of every pass of a fixed-length row (Stockham,
    one pad float2 per 16): pass 0 writes butterfly b's outputs at
    spad2(b R + r); a later pass reads spad2(b + r N/R) and writes
    spad2(q Ns R + k + r Ns) (k = b mod Ns, q = b / Ns); the epilogue reads
    spad2(o), o = j + i T.  With consecutive threads on consecutive b, no
    half-warp's 64-bit accesses meet a bank twice when the first radix is 16
    and every later N/R and Ns is a multiple of 16 (the fused workload's
    10000 = 16 x 25 x 25 among them).  Other schedules are not: a first
    radix R places consecutive threads' outputs about 17 R / 16 slots apart
    (10000 is conflict-free, 12288 = 32 x 16 x 24 two-way, 15000 =
    10 x 10 x 10 x 15 five-way in its first pass)."""
    lanes = np.arange(T)
    warps = [lanes[w:w + 32] for w in range(0, T, 32)]
    Ns = 1
    for p, R in enumerate(radices):
        nb = N // R
        gm = max(1, 32 // R)
        for g in range(gm):
            for warp in warps:
                b = warp + g * T
                live = b < nb
                for r in range(R):
                    if p == 0:
                        wr = [spad2(int(x) * R + r) if ok else None for x, ok in zip(b, live)]
                        assert _half_warp_degree(wr) == 1, (p, g, r)
                        continue
                    rd = [spad2(int(x) + r * nb) if ok else None for x, ok in zip(b, live)]
                    q, k = b // Ns, b % Ns
                    wr = [spad2(int(qq) * Ns * R + int(kk) + r * Ns) if ok else None
                          for qq, kk, ok in zip(q, k, live)]
                    assert _half_warp_degree(rd) == 1, ("read", p, g, r)
                    assert _half_warp_degree(wr) == 1, ("write", p, g, r)
        Ns *= R
    for i in range(-(-N // T)):
        for warp in warps:
            o = warp + i * T
            assert _half_warp_degree([spad2(int(x)) if x < N else None for x in o]) == 1


@pytest.mark.parametrize("N,T,radices,first", [(12288, 512, (32, 16, 24), 2), (15000, 512, (10, 10, 10, 15), 5),
                                                (7000, 288, (28, 10, 25), 3)])
def test_first_pass_write_conflicts(N, T, radices, first):
    """The first-pass writes of a radix that is not 16 meet a bank `first`
    times in some half-warp (the model of the test above)."""
    R = radices[0]
    b = np.arange(T)
    worst = max(_half_warp_degree([spad2(int(x) * R + r) if x < N // R else None for x in b[w:w + 32]])
                for w in range(0, T, 32) for r in range(R))
    assert worst == first
