"""The FP32 screen of the FP64 acceptance rule (Eq. 8), in the threshold form the
block scan evaluates, checked on the CPU (no GPU).

FP64 and FX64 modes decide every attempt by the exact rule: accept if dE <= 0
or u < exp(-beta c dE).  The scan first screens each lane in FP32 and applies
the exact rule only where the screen is unsure, so the decisions are the exact
rule's as long as no sure verdict is wrong.  Per lane and block, with every
operation rounded to float32 as on the device:

    r  = 1 / cb
    dA = (nlu (1 - 2e-6) - cb errd - 2e-6) r (1 - 2e-6),   dAe = max(dA, errd)
    dR = (nlu (1 + 2e-6) + cb errd + 2e-6) r (1 + 2e-6)
    sure accept:  d32 <= -errd,  or  errd <= d32 < dAe
    sure reject:  d32 > dR
    unsure:       -errd < d32 < errd,  or  dAe <= d32 <= dR

where nlu is -ln u in float32 (from the same Philox words as the exact u), cb
= float32(beta c), and d32 is the FP32 field difference, within errd / 2 of
the exact one (errd = 2.4e-5 Jtot bounds the conversion and up to 64 FP32
corrections with a factor 2 to spare).  The test draws differences on and
around the decision boundary and asserts that no sure verdict disagrees with
the exact rule, with the thresholds also moved one float32 step towards the
sure side (covering another order of the device's roundings or a logf one
step off).
"""
import numpy as np

f32 = np.float32


def _nlu32(ux1, ux2):
    # the device's FP64-mode -ln u in float32: u from the words' top 32 and
    # next 21 bits, as in the proposal draw
    uf = ux1.astype(f32) * f32(2.0 ** -32) + ((ux2 >> np.uint32(11)) + np.uint32(1)).astype(f32) * f32(2.0 ** -53)
    return (-np.log(uf)).astype(f32)


def _unit53(ux1, ux2):
    bits = ((ux1.astype(np.uint64) << np.uint64(32)) | ux2.astype(np.uint64)) >> np.uint64(11)
    return (bits + np.uint64(1)).astype(np.float64) * 2.0 ** -53


def _screen(d32, cb32, nlu32, errd32):
    one = f32(1.0)
    k = f32(2e-6)
    r = (one / cb32).astype(f32)
    dA = ((((nlu32 * (one - k)).astype(f32) - (cb32 * errd32).astype(f32)).astype(f32) - k).astype(f32) * r).astype(f32)
    dA = (dA * (one - k)).astype(f32)
    dR = ((((nlu32 * (one + k)).astype(f32) + (cb32 * errd32).astype(f32)).astype(f32) + k).astype(f32) * r).astype(f32)
    dR = (dR * (one + k)).astype(f32)
    return dA, dR


def _verdicts(d32, dA, dR, errd32):
    dAe = np.maximum(dA, errd32)
    unsure = ((d32 > -errd32) & (d32 < errd32)) | ((d32 >= dAe) & (d32 <= dR))
    vote = d32 <= dR
    return vote & ~unsure, ~vote  # sure accept, sure reject


def _cases(rng, n, jtot, c):
    ux1 = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    ux2 = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    # a tenth of the draws with u within 2^-20 of 1 (-ln u tiny)
    near1 = rng.random(n) < 0.1
    ux1[near1] = np.uint32(0xFFFFFFFF) - rng.integers(0, 4096, size=near1.sum()).astype(np.uint32)
    u = _unit53(ux1, ux2)
    T = jtot * np.exp(rng.uniform(np.log(0.002), np.log(5.0), size=n))
    cb64 = c / T
    dstar = -np.log(u) / cb64  # the exact rule's boundary
    errd = 2.4e-5 * jtot
    kind = rng.integers(0, 4, size=n)
    d64 = np.where(kind == 0, dstar * (1.0 + rng.uniform(-1e-4, 1e-4, size=n)),            # on the boundary
          np.where(kind == 1, dstar + rng.uniform(-2.0, 2.0, size=n) * errd,                 # within a few errd
          np.where(kind == 2, rng.uniform(-2.0, 2.0, size=n) * errd,                         # around dE = 0
                   rng.uniform(-3.0, 3.0, size=n) * jtot)))                                  # anywhere
    d32 = (d64 + rng.uniform(-0.5, 0.5, size=n) * errd).astype(f32)
    return ux1, ux2, u, cb64, d64, d32, f32(errd)


def test_screen_sure_verdicts_agree_with_the_exact_rule():
    rng = np.random.default_rng(20240531)
    nsure = ntot = 0
    for jtot in (0.7, 6.0, 55.0):
        for c in (1.0, 2.0):
            ux1, ux2, u, cb64, d64, d32, errd32 = _cases(rng, 200_000, jtot, c)
            with np.errstate(over="ignore"):  # exp(+large) = inf: accept, as the rule says
                exact = (d64 <= 0.0) | (u < np.exp(-cb64 * d64))
            cb32 = cb64.astype(f32)
            nlu = _nlu32(ux1, ux2)
            for dn in (-1, 0, 1):  # logf one float32 step either way
                nlu_v = nlu if dn == 0 else np.nextafter(nlu, f32(dn * np.inf)).astype(f32)
                dA, dR = _screen(d32, cb32, nlu_v, errd32)
                for dA_t, dR_t in ((dA, dR), (np.nextafter(dA, f32(np.inf)), np.nextafter(dR, f32(-np.inf)))):
                    acc, rej = _verdicts(d32, dA_t.astype(f32), dR_t.astype(f32), errd32)
                    bad_acc = np.flatnonzero(acc & ~exact)
                    bad_rej = np.flatnonzero(rej & exact)
                    assert bad_acc.size == 0, (jtot, c, d64[bad_acc[:3]], d32[bad_acc[:3]], u[bad_acc[:3]])
                    assert bad_rej.size == 0, (jtot, c, d64[bad_rej[:3]], d32[bad_rej[:3]], u[bad_rej[:3]])
                    nsure += int(acc.sum() + rej.sum())
                    ntot += acc.size
    # the screen decides most draws even on this boundary-heavy mix
    assert nsure > 0.5 * ntot


def test_screen_degenerate_cases():
    """u = 1 (-ln u = 0): the exact rule accepts exactly dE <= 0, and the
    screen is sure only outside the margin; very hot and very cold slots keep
    dR above errd and the unsure band ordered."""
    errd = f32(2.4e-5 * 6.0)
    for cb in (f32(1e-6), f32(0.01), f32(1.0), f32(1e4), f32(1e7)):
        for nlu in (f32(0.0), f32(1e-12), f32(0.7), f32(36.7)):
            d = np.array([-1.0, -errd, -errd / 2, 0.0, errd / 2, errd, 2 * errd, 10.0], dtype=f32)
            dA, dR = _screen(d, np.full_like(d, cb), np.full_like(d, nlu), errd)
            assert np.all(dR > errd)
            acc, rej = _verdicts(d, dA, dR, errd)
            assert not np.any(acc & rej)
            # sure accepts need dE < 0 for -ln u = 0
            if nlu == 0.0:
                assert np.all(d[acc] <= -errd)
