"""Host-side models of the 16384- and 2048-point class-local schedules of the
correlate's occupancy form (the shared-memory slots, thread -> butterfly map,
exchange groups and output order written in csrc/fft.cuh and
csrc/xcorr_tm.cu), checked without a GPU:

* the model's transform, pass by pass through the padded slots, equals the
  inverse DFT (numpy) -- so the addresses, twiddle exponents and output order
  are those of a Stockham radix 16-16-16-4 (16-16-8) inverse transform;
* each in-place exchange writes exactly the slots its synchronising group
  read (the class pair's four warps; the four lanes of one residue, which
  share a warp), so the named barrier and __syncwarp guard every reuse;
* every slot offset from a thread's base is carry-free (a compile-time
  constant in the kernel), and every access stays below the buffer size;
* every warp access of the schedule puts each half-warp on 16 distinct
  8-byte bank pairs (no shared-memory bank conflicts).
"""
import numpy as np

N, T = 16384, 1024
SMEM = N + N // 16 + N // 256 + N // 4096


def pad_q(i):
    return i + (i >> 4) + (i >> 8) + (i >> 12)


def q_off(d):
    return d + d // 16 + d // 256 + d // 4096


def perm(t):
    p = t & 63
    ip = (p & 1) | (((p >> 5) & 1) << 1) | (((p >> 1) & 3) << 2) | (((p >> 4) & 1) << 4) | (((p >> 3) & 1) << 5)
    return (t >> 6) + 16 * ip


def quad_m(jp, i):
    return (jp & 255) + 256 * ((jp >> 8) + 4 * i)


def out_index(jp, r):
    return quad_m(jp, r >> 2) + 4096 * (r & 3)


JP = [perm(t) for t in range(T)]


def _dft(u):
    """Inverse-direction DFT of the rows of u (unscaled)."""
    R = u.shape[-1]
    k = np.arange(R)
    return u @ np.exp(2j * np.pi * np.outer(k, k) / R)


def _w(M, e):
    return np.exp(2j * np.pi * np.asarray(e) / M)


def test_thread_map_is_a_bijection_and_classes_sit_on_their_warps():
    assert sorted(JP) == list(range(T))
    for t in range(T):
        assert JP[t] % 16 == t // 64  # class c on threads 64 c .. 64 c + 63 (warps 2c, 2c + 1)


def test_model_equals_inverse_dft_and_exchanges_stay_in_their_groups():
    rng = np.random.default_rng(16384)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    buf = np.full(SMEM, np.nan, complex)
    t_all = np.arange(T)
    v = x[t_all[:, None] + T * np.arange(16)[None, :]]  # thread t holds x[t + T r]
    # pass 1 (NS = 1, butterfly J = t) and the first-pass stores at 16 t + u
    v = _dft(v)
    for t in range(T):
        base = pad_q(16 * t)
        assert [base + u for u in range(16)] == [pad_q(16 * t + u) for u in range(16)]
        buf[base:base + 16] = v[t]
    # class gathers x[jp + T r], pass 2 (NS = 16), class stores
    read = {}
    for t in range(T):
        g = [pad_q(JP[t]) + q_off(T * r) for r in range(16)]
        assert g == [pad_q(JP[t] + T * r) for r in range(16)] and max(g) < SMEM
        v[t] = buf[g]
        read.setdefault(t >> 7, set()).update(g)
    k2 = np.array(JP) % 16
    v = _dft(v * _w(256, np.outer(k2, np.arange(16))))
    wrote = {}
    for t in range(T):
        jp = JP[t]
        base = pad_q((jp >> 4) * 256 + (jp & 15))
        s = [base + q_off(16 * u) for u in range(16)]
        assert s == [pad_q((jp >> 4) * 256 + (jp & 15) + 16 * u) for u in range(16)]
        buf[s] = v[t]
        wrote.setdefault(t >> 7, set()).update(s)
    assert read == wrote  # the class pair's warps overwrite only what they read
    # gathers, pass 3 (NS = 256), the quad stores
    for t in range(T):
        v[t] = buf[[pad_q(JP[t]) + q_off(T * r) for r in range(16)]]
    k3 = np.array(JP) % 256
    v = _dft(v * _w(4096, np.outer(k3, np.arange(16))))
    qread, qwrote = {}, {}
    for t in range(T):
        jp = JP[t]
        h, k = jp >> 8, jp & 255
        qread.setdefault((t >> 5, k), set()).update(pad_q(jp + T * r) for r in range(16))
        base = pad_q(4096 * h + k)
        s = [base + q_off(256 * u) for u in range(16)]
        assert s == [pad_q(4096 * h + k + 256 * u) for u in range(16)]
        buf[s] = v[t]
        qwrote.setdefault((t >> 5, k), set()).update(s)
    assert qread == qwrote and all(len(s) == 64 for s in qread.values())  # four lanes of one warp
    # quad gathers and the radix-4 pass (NS = 4096)
    out = np.full(N, np.nan, complex)
    for t in range(T):
        jp = JP[t]
        h, k = jp >> 8, jp & 255
        base = pad_q(k + 256 * h)
        vv = np.empty(16, complex)
        for i in range(4):
            for s in range(4):
                a = base + q_off(1024 * i + 4096 * s)
                assert a == pad_q(k + 256 * h + 1024 * i + 4096 * s) and a < SMEM
                vv[4 * i + s] = buf[a]
        for i in range(4):
            m = quad_m(jp, i)
            vv[4 * i:4 * i + 4] = _dft(vv[4 * i:4 * i + 4] * _w(N, m * np.arange(4)))
        for r in range(16):
            o = out_index(jp, r)
            assert o % 256 == jp % 256  # the row statistics' period-256 shortcut
            out[o] = vv[r]
    ref = np.fft.ifft(x) * N
    assert not np.isnan(out).any()
    assert np.abs(out - ref).max() <= 1e-9 * np.abs(ref).max()


def _wavefronts(slots):
    n = 0
    for half in (slots[:16], slots[16:]):
        pairs = {}
        for a in set(half):
            pairs.setdefault(a % 16, set()).add(a)
        n += max(len(s) for s in pairs.values())
    return n


def test_every_warp_access_is_free_of_bank_conflicts():
    warps = [range(w * 32, w * 32 + 32) for w in range(T // 32)]
    pats = {
        "first-pass stores": lambda t, a: 16 * t + a,
        "class gathers": lambda t, a: JP[t] + T * a,
        "class stores": lambda t, a: 256 * (JP[t] >> 4) + (JP[t] & 15) + 16 * a,
        "quad stores": lambda t, a: 4096 * (JP[t] >> 8) + (JP[t] & 255) + 256 * a,
        "quad gathers": lambda t, a: quad_m(JP[t], a >> 2) + 4096 * (a & 3),
    }
    for name, f in pats.items():
        for ws in warps:
            for a in range(16):
                assert _wavefronts([pad_q(f(t, a)) for t in ws]) == 2, (name, ws[0], a)


# --- N = 2048: radix 16-16-8, T = 128, classes on 8 lanes of one warp --------
N2, T2 = 2048, 128
SMEM2 = N2 + N2 // 8 + N2 // 128


def pad_2k(e):
    return e + (e >> 3) + (e >> 7)


def off_2k(d):
    return d + d // 8 + d // 128


def perm_2k(t):
    c = (t & 3) | (((t >> 5) & 3) << 2)
    i = ((t >> 4) & 1) | (((t >> 2) & 3) << 1)
    return c + 16 * i


JP2 = [perm_2k(t) for t in range(T2)]


def test_2048_map_is_a_bijection_with_each_class_in_one_warp():
    assert sorted(JP2) == list(range(T2))
    warps = {}
    for t in range(T2):
        warps.setdefault(JP2[t] % 16, set()).add(t >> 5)
    assert all(len(w) == 1 for w in warps.values()) and len(warps) == 16


def test_2048_model_equals_inverse_dft_and_classes_stay_in_their_warp():
    rng = np.random.default_rng(2048)
    x = rng.standard_normal(N2) + 1j * rng.standard_normal(N2)
    buf = np.full(SMEM2, np.nan, complex)
    t_all = np.arange(T2)
    v = _dft(x[t_all[:, None] + T2 * np.arange(16)[None, :]])  # pass 1, NS = 1
    for t in range(T2):
        s = [pad_2k(16 * t) + off_2k(u) for u in range(16)]
        assert s == [pad_2k(16 * t + u) for u in range(16)]
        buf[s] = v[t]
    read = {}
    for t in range(T2):
        g = [pad_2k(JP2[t]) + off_2k(T2 * r) for r in range(16)]
        assert g == [pad_2k(JP2[t] + T2 * r) for r in range(16)] and max(g) < SMEM2
        v[t] = buf[g]
        read.setdefault((t >> 5, JP2[t] % 16), set()).update(g)
    v = _dft(v * _w(256, np.outer(np.array(JP2) % 16, np.arange(16))))  # NS = 16
    wrote = {}
    for t in range(T2):
        jp = JP2[t]
        base = pad_2k((jp >> 4) * 256 + (jp & 15))
        s = [base + off_2k(16 * u) for u in range(16)]
        assert s == [pad_2k((jp >> 4) * 256 + (jp & 15) + 16 * u) for u in range(16)]
        buf[s] = v[t]
        wrote.setdefault((t >> 5, jp % 16), set()).update(s)
    assert read == wrote  # the class's lanes (one warp) overwrite only what they read
    for t in range(T2):
        v[t] = buf[[pad_2k(JP2[t]) + off_2k(T2 * r) for r in range(16)]]
    out = np.full(N2, np.nan, complex)
    for t in range(T2):
        jp = JP2[t]
        for q in range(2):  # radix-8 butterflies J = jp + 128 q (NS = 256): inputs v[q + 2 s]
            J = jp + 128 * q
            u = _dft(v[t][q::2] * _w(2048, J * np.arange(8)))
            for k in range(8):
                out[J + 256 * k] = u[k]  # = X[jp + 128 (q + 2 k)]
    ref = np.fft.ifft(x) * N2
    assert not np.isnan(out).any()
    assert np.abs(out - ref).max() <= 1e-9 * np.abs(ref).max()


def test_2048_every_warp_access_is_free_of_bank_conflicts():
    pats = {
        "first-pass stores": lambda t, a: 16 * t + a,
        "class gathers": lambda t, a: JP2[t] + T2 * a,
        "class stores": lambda t, a: 256 * (JP2[t] >> 4) + (JP2[t] & 15) + 16 * a,
    }
    for name, f in pats.items():
        for w in range(T2 // 32):
            for a in range(16):
                assert _wavefronts([pad_2k(f(t, a)) for t in range(w * 32, w * 32 + 32)]) == 2, (name, w, a)
