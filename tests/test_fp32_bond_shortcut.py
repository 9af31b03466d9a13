"""The FP32 n-vector bond shortcut's margins (host-side check of the
arithmetic in vec_local_kernel).

A positive FP32 bond with y = K2 p_i p_j is on iff its 32-bit uniform w is
below floor(p 2^32), p = -expm1f(-y).  The kernel first compares y with
bounds derived from the top byte b of w: on whatever the low bits if
y > yhi (1 + 1e-4) + 1e-6 with yhi = -log(1 - (b + 1)/256), off if
y < ylo (1 - 1e-4) - 1e-6 with ylo = -log(1 - b/256), both logs taken with
the fast single-precision log.  That must never contradict the exact FP32
rule, for any expm1f result within 1 ulp and any fast-log result within
its documented error (2^-21.41 absolute on [0.5, 2], 3 ulp elsewhere),
which is what this test checks over every byte and a dense set of y around
each byte's edges."""
import numpy as np

F = np.float32


def ulp_shift(x, k):
    """x moved by k units in the last place (float32)."""
    x = np.asarray(x, dtype=np.float32)
    for _ in range(abs(k)):
        x = np.nextafter(x, np.float32(np.inf) if k > 0 else np.float32(-np.inf)).astype(np.float32)
    return x


def thr_of(p):
    """floor(p 2^32), 2^32 for p >= 1, 0 for p <= 0 (the kernel's threshold)."""
    p = np.asarray(p, dtype=np.float64)
    t = np.floor(np.clip(p, 0, 1) * 2.0 ** 32)
    return np.where(p >= 1, 2.0 ** 32, t)


def test_shortcut_never_contradicts_the_exact_rule():
    rng = np.random.default_rng(0)
    for b in range(256):
        lo_true = -np.log1p(-b / 256.0)
        hi_true = -np.log1p(-(b + 1) / 256.0) if b < 255 else np.inf
        # the fast log's documented error: 2^-21.41 absolute for arguments
        # in [0.5, 2], else 3 ulp
        for dlog in (-1, 0, 1):
            def fast_log_bound(k):
                x = F(1.0) - F(k) * F(1 / 256)
                v = F(-np.log(x))
                if x >= 0.5:
                    return F(v + dlog * 2.0 ** -21.41)
                return ulp_shift(v, 3 * dlog)
            ylo = fast_log_bound(b) if b > 0 else F(-0.0)
            yhi = fast_log_bound(b + 1) if b < 255 else F(np.inf)
            on_bound = yhi * F(1.0001) + F(1e-6)
            off_bound = ylo * F(0.9999) - F(1e-6)
            # y just beyond the shortcut bounds, and random y around the edges
            cand = [ulp_shift(on_bound, 1), ulp_shift(on_bound, 4), ulp_shift(off_bound, -1), ulp_shift(off_bound, -4)]
            span = [lo_true * 0.99 - 1e-5, (hi_true if np.isfinite(hi_true) else lo_true + 10) * 1.01 + 1e-5]
            cand += list(rng.uniform(max(span[0], 1e-9), span[1], 200).astype(np.float32))
            for y in cand:
                y = F(y)
                if not np.isfinite(y) or y <= 0:
                    continue
                p = F(-np.expm1(-np.float64(y)))
                for dp in (-1, 0, 1):
                    t = thr_of(ulp_shift(p, dp))
                    if y > on_bound:
                        assert t >= (b + 1) * 2.0 ** 24, (b, y)  # every w with top byte b is below t
                    if y < off_bound:
                        assert t <= b * 2.0 ** 24, (b, y)  # no such w is below t


def test_shortcut_leaves_only_a_narrow_band_to_the_exact_path():
    # the fraction of uniformly drawn (y, b) pairs that fall between the
    # bounds is about 1/256 plus the margins
    rng = np.random.default_rng(1)
    y = rng.uniform(0.01, 4.0, 20000).astype(np.float32)
    b = rng.integers(0, 256, 20000)
    ylo = -np.log(F(1.0) - b.astype(np.float32) / F(256))
    yhi = np.where(b < 255, -np.log(np.maximum(F(1.0) - (b + 1).astype(np.float32) / F(256), F(1e-30))), np.inf)
    exact = ~((y > yhi * F(1.0001) + F(1e-6)) | (y < ylo * F(0.9999) - F(1e-6)))
    assert exact.mean() < 0.02
