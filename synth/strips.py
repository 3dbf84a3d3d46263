"""Synthetic silicon-strip raw data for the clustering step (Sec. 4): per
module N strips with a pedestal-subtracted Gaussian noise of 2-6 ADC counts,
about 1 % bad strips, and signal hits whose charge (log-normal around ~110 ADC
counts, long upper tail) is shared by neighbouring strips with a Gaussian
profile.  No clustering arithmetic lives here."""
import numpy as np


def make_strip_calibration(n_modules, n_strips, rng, bad_frac=0.01):
    """noise_q [M, N] uint16 = round(8 x noise), bad [M, N] uint8."""
    noise = rng.uniform(2.0, 6.0, (n_modules, n_strips))
    noise_q = np.round(8.0 * noise).astype(np.uint16)
    bad = (rng.random((n_modules, n_strips)) < bad_frac).astype(np.uint8)
    return noise_q, bad


def make_strip_event(noise_q, rng, occupancy=0.01, width=(0.3, 0.9)):
    """adc [M, N] uint16 (10-bit) for one event on the given calibration."""
    M, N = noise_q.shape
    sigma = noise_q.astype(np.float64) / 8.0
    adc = rng.normal(0.0, 1.0, (M, N)) * sigma
    n_hits = int(occupancy * M * N / 3)
    mod = rng.integers(0, M, n_hits)
    x = rng.uniform(0.0, N, n_hits)
    q = rng.lognormal(np.log(110.0), 0.35, n_hits)
    w = rng.uniform(width[0], width[1], n_hits)
    base = np.floor(x).astype(np.int64)
    for d in range(-3, 4):
        s = base + d
        ok = (s >= 0) & (s < N)
        c = s + 0.5 - x
        frac = np.exp(-0.5 * (c / w) ** 2) / (np.sqrt(2 * np.pi) * w)
        np.add.at(adc, (mod[ok], s[ok]), (q * frac)[ok])
    return np.clip(np.round(adc), 0, 1023).astype(np.uint16)
