"""The operand-precision reasoning of the tensor form, checked on CPU.

The tensor form evaluates the pair sum of Eq. (HP) through Eq. (taylor)
regrouped by harmonic, S(f) = sum_n a_n (c_n^T W c_n + s_n^T W s_n), as
products W' Z with 16-bit operands (W' the upper triangle of W with the
off-diagonal part doubled, Z = a_n (cos, sin)(n theta)) and FP32 weights x
in the final dot product.  This model rounds the operands exactly as the
kernels do (round to nearest even; BF16 hi + lo splits) and evaluates the
products in FP64, so that only the operands' rounding differs from the same
truncated series in FP64.  It pins the choices the kernels make: FP16
operands stay well within 1e-3 of the peak, BF16 with W' split and Z single
does not do much better than FP16, and BF16 with both operands split (three
of the four hi/lo products) removes the rounding to ~1e-5 and below.
"""
import numpy as np
import pytest

import synth

sp = pytest.importorskip("scipy.special")


def to_bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def to_fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float64)


def split(x, r):
    hi = r(x)
    return hi, r(np.asarray(x, np.float32).astype(np.float64) - hi)


def model(t, Wp, freqs, a, mode):
    """Peak-normalised periodogram of the truncated series with the given operand treatment."""
    n = np.arange(1, len(a) + 1)
    if mode == "fp16":
        Wq = [to_fp16(Wp)]
    elif mode == "exact":
        Wq = [Wp]
    else:
        Wq = list(split(Wp, to_bf16))                # BF16 W': hi + lo
    out = []
    for f in freqs:
        th = 2.0 * np.pi * ((f * t) % 1.0)
        X = np.concatenate([np.cos(np.outer(th, n)), np.sin(np.outer(th, n))], axis=1)   # x (FP32 in the epilogue)
        Z = X * np.concatenate([a, a])[None, :]
        if mode == "exact":
            D = Wq[0] @ Z
        elif mode == "fp16":
            D = Wq[0] @ to_fp16(Z)
        elif mode == "bf16 w split":
            zq = to_bf16(Z)
            D = Wq[0] @ zq + Wq[1] @ zq
        else:                                        # "bf16 split": W' hi x (Z hi + lo) + W' lo x Z hi
            zh, zl = split(Z, to_bf16)
            D = Wq[0] @ (zh + zl) + Wq[1] @ zh
        out.append(np.sum(np.asarray(X, np.float32).astype(np.float64) * D))
    return np.array(out)


@pytest.mark.parametrize("seed,sigma_t,n_max", [(3, 0.3, 16), (7, 0.45, 12)])
def test_operand_rounding_of_the_tensor_form(seed, sigma_t, n_max):
    b = synth.ragged_batch(1, seed=seed, n_lo=300, n_hi=420)
    t, m, e = b.curve(0)
    t = t - t.min()
    y = m.astype(np.float64)
    sy = float(np.median(e.astype(np.float64)))
    g = np.exp(-np.subtract.outer(y, y) ** 2 / (2.0 * sy * sy))
    W = g - g.mean()                                   # zero sum, as W = G - IP (Eq. (IP))
    Wp = np.triu(W, 1) * 2.0 + np.diag(np.diag(W))
    kap = 1.0 / sigma_t ** 2
    a = 2.0 * sp.ive(np.arange(1, n_max + 1), kap)     # a_n = 2 e^-k I_n(k)
    freqs = np.linspace(0.05, 2.0, 40)
    ref = model(t, Wp, freqs, a, "exact")
    # the truncated series itself is the pair sum of Eq. (HP) to within its tail
    direct = np.array([np.sum(W * np.exp(-2.0 * np.sin(np.pi * f * np.subtract.outer(t, t)) ** 2 / sigma_t ** 2))
                       for f in freqs])
    scale = np.max(np.abs(direct))
    assert np.max(np.abs(ref - direct)) <= 1e-3 * scale
    err = {m_: np.max(np.abs(model(t, Wp, freqs, a, m_) - ref)) / scale
           for m_ in ("fp16", "bf16 w split", "bf16 split")}
    print("\nsigma_t %.2f, %d harmonics: peak-relative operand-rounding error" % (sigma_t, n_max),
          {k: "%.2e" % v for k, v in err.items()})
    assert err["fp16"] <= 1e-3
    assert err["bf16 split"] <= 2e-5
    assert err["bf16 w split"] > 10.0 * err["bf16 split"]       # Z's single BF16 rounding dominates
    assert err["bf16 w split"] > 0.5 * err["fp16"]              # 8 significand bits in Z against 11
