"""Pins for the FP64 oracle: each test checks an oracle routine against
something other than itself -- a direct O(N^2) sum, an independent library,
a closed form from the literature, an invariant or a statistical law -- so
that a dropped term, a wrong sign or index, or a transposed operand fails.

Paper: arXiv:0906.4175, Sec. 1.1, Eqs. (1)-(4).
"""
import math
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


# ---------------------------------------------------------------- FFT ------

@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 64, 256, 1024])
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_direct_dft(oracle_lib, N, sign):
    """Own radix-2 FFT == the O(N^2) definition sum_n x_n exp(sign 2 pi i nk/N)."""
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    n = np.arange(N)
    W = np.exp(sign * 2j * np.pi * np.outer(n, n) / N)
    ref = W @ x
    got = oracle_lib.fft(x, sign)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1, N) * np.max(np.abs(x))


def test_fft_matches_numpy_large(oracle_lib):
    """Against an independent library (numpy pocketfft) at N = 2^16."""
    rng = np.random.default_rng(7)
    N = 1 << 16
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    assert np.max(np.abs(oracle_lib.fft(x, -1) - np.fft.fft(x))) < 1e-9
    assert np.max(np.abs(oracle_lib.fft(x, +1) - N * np.fft.ifft(x))) < 1e-9


def test_fft_parseval_and_roundtrip(oracle_lib):
    rng = np.random.default_rng(3)
    N = 1 << 12
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = oracle_lib.fft(x, -1)
    assert abs(np.sum(np.abs(X) ** 2) / N - np.sum(np.abs(x) ** 2)) < 1e-9 * np.sum(np.abs(x) ** 2)
    back = oracle_lib.fft(X, +1) / N
    assert np.max(np.abs(back - x)) < 1e-12


def test_fft_rejects_non_power_of_two(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.fft(np.ones(12), -1)


# ---------------------------------------------------------------- PSD ------

def test_psd_eq2_special_values(oracle_lib):
    """Eq. (2): at f = f0 every power of x is 1, so S = 4.49^-56 + 0.16 + 0.52 + 0.32;
    the coefficients are the ones the paper prints (golden fixture)."""
    g = _golden_constants()
    f0 = g["psd_f0_hz"]
    expect = g["psd_c1"] ** g["psd_p1"] + g["psd_c2"] + g["psd_c3"] + g["psd_c4"]
    assert abs(oracle_lib.psd_eq2(f0) - expect) < 1e-15
    # doubling f at high frequency: the x^2 term dominates -> S(2f)/S(f) -> 4
    f = 2.0e5
    r = oracle_lib.psd_eq2(2 * f) / oracle_lib.psd_eq2(f)
    assert abs(r - 4.0) < 1e-5
    # scale: S0 multiplies the whole curve
    assert abs(oracle_lib.psd_eq2(200.0, 150.0, 9e-46) / oracle_lib.psd_eq2(200.0) - 9e-46) < 1e-60


def test_psd_eq2_logslopes(oracle_lib):
    """Local power-law index d ln S / d ln f: -56 deep in the seismic wall,
    +2 at high frequency (each coefficient's exponent, Eq. 2)."""
    def slope(f):
        h = 1e-6
        return (math.log(oracle_lib.psd_eq2(f * (1 + h))) - math.log(oracle_lib.psd_eq2(f * (1 - h)))) / (
            math.log(1 + h) - math.log(1 - h))
    assert abs(slope(5.0) + 56.0) < 1e-6
    assert abs(slope(1.0e6) - 2.0) < 1e-4
    # where the seismic term is negligible and x is small, the -4.52 term leads:
    # slope = -4.52 * w + 2 * (1 - w - c) with weights of each term
    f = 60.0
    x = f / 150.0
    t2, t3, t4 = 0.16 * x ** -4.52, 0.52, 0.32 * x * x
    pred = (-4.52 * t2 + 2 * t4) / (t2 + t3 + t4)
    assert abs(slope(f) - pred) < 1e-6


# ----------------------------------------------------------- template ------

def _tau_2pn(m1, m2, f):
    """2PN time to coalescence at GW frequency f (standard form; e.g.
    Blanchet et al. 1996 / Sathyaprakash & Dhurandhar), independent of Psi."""
    M = (m1 + m2) * 4.925490947e-6
    eta = m1 * m2 / (m1 + m2) ** 2
    v = (math.pi * M * f) ** (1.0 / 3.0)
    return (5.0 * M / (256.0 * eta * v ** 8)) * (
        1.0 + (743.0 / 252.0 + 11.0 * eta / 3.0) * v ** 2 - (32.0 * math.pi / 5.0) * v ** 3
        + (3058673.0 / 508032.0 + 5429.0 * eta / 504.0 + 617.0 * eta ** 2 / 72.0) * v ** 4)


@pytest.mark.parametrize("m1,m2", [(1.0, 1.0), (1.4, 1.4), (1.2, 2.9), (10.0, 1.5), (20.0, 15.0)])
@pytest.mark.parametrize("f", [40.0, 97.3, 250.0, 700.0])
def test_psi_stationary_phase_time(oracle_lib, m1, m2, f):
    """Stationary phase: dPsi/df = -2 pi tau(f) with tau the 2PN time to
    coalescence -- every phase coefficient (and the 3/(128 eta) prefactor)
    enters this relation."""
    if f >= oracle_lib.f_isco(m1, m2):
        pytest.skip("above ISCO")
    h = f * 1e-5
    d = (oracle_lib.psi(m1, m2, f + h) - oracle_lib.psi(m1, m2, f - h)) / (2 * h)
    # 4th-order central difference to beat truncation error
    d4 = (8 * (oracle_lib.psi(m1, m2, f + h) - oracle_lib.psi(m1, m2, f - h))
          - (oracle_lib.psi(m1, m2, f + 2 * h) - oracle_lib.psi(m1, m2, f - 2 * h))) / (12 * h)
    tau = _tau_2pn(m1, m2, f)
    assert abs(d4 + 2 * math.pi * tau) < 1e-6 * 2 * math.pi * tau
    assert abs(d + 2 * math.pi * tau) < 1e-4 * 2 * math.pi * tau


def test_psi_newtonian_limit(oracle_lib):
    """As v -> 0 the Newtonian term 3/(128 eta v^5) dominates Psi."""
    m1, m2 = 1.4, 1.4
    M = (m1 + m2) * 4.925490947e-6
    eta = 0.25
    f = 1e-6
    v = (math.pi * M * f) ** (1 / 3)
    lead = 3.0 / (128.0 * eta * v ** 5)
    assert abs(oracle_lib.psi(m1, m2, f) / lead - 1.0) < 1e-3


def test_newtonian_chirp_time(oracle_lib):
    """A 1+1 Msun binary spends ~43.5 s above 40 Hz at Newtonian order:
    tau_0 = 5/256 (pi f)^(-8/3) Mc^(-5/3)."""
    Mc = (1.0 * 1.0) ** 0.6 / 2.0 ** 0.2 * 4.925490947e-6
    tau0 = 5.0 / 256.0 * (math.pi * 40.0) ** (-8.0 / 3.0) * Mc ** (-5.0 / 3.0)
    assert 43.0 < tau0 < 44.0
    # the oracle's phase slope at 40 Hz equals 2 pi tau_2PN, within 2PN corrections of tau0
    h = 1e-3
    slope = -(oracle_lib.psi(1.0, 1.0, 40.0 + h) - oracle_lib.psi(1.0, 1.0, 40.0 - h)) / (2 * h) / (2 * math.pi)
    assert 0.9 * tau0 < slope < 1.1 * tau0


@pytest.mark.parametrize("m1,m2", [(1.0, 1.0), (3.0, 3.0), (17.5, 17.5)])
def test_isco_frequency_from_kepler(oracle_lib, m1, m2):
    """f_isco is twice the Keplerian orbital frequency at r = 6M:
    f = 2 * sqrt(M / r^3) / (2 pi) with G = c = 1."""
    M = (m1 + m2) * 4.925490947e-6
    r = 6.0 * M
    f_kepler_gw = 2.0 * math.sqrt(M / r ** 3) / (2.0 * math.pi)
    assert abs(oracle_lib.f_isco(m1, m2) / f_kepler_gw - 1.0) < 1e-14
    if m1 + m2 == 2.0:
        assert 2198.0 < f_kepler_gw < 2200.0
    if m1 + m2 == 35.0:
        assert 125.0 < f_kepler_gw < 126.0


def test_band_rule(oracle_lib):
    """Sec. 1.1: 40 Hz up to min(Nyquist, f_isco); 2^20 points at 4096 Hz."""
    g = _golden_constants()
    N, fs = int(g["segment_points"]), g["fs_hz"]
    assert N / fs == g["segment_seconds"]
    lo, hi = oracle_lib.band(N, fs, g["f_low_hz"], 1e9)
    assert lo == 40 * 256 and hi == N // 2          # f_low exactly on a bin is included; Nyquist excluded
    lo, hi = oracle_lib.band(N, fs, 40.0, 733.0)    # f_cut exactly on a bin is included
    assert hi == 733 * 256 + 1
    lo, hi = oracle_lib.band(N, fs, 40.0, 733.001)
    assert hi == 733 * 256 + 1
    lo, hi = oracle_lib.band(1024, 1024.0, 40.3, 100.0)
    assert lo == 41 and hi == 101


def test_htilde_amplitude_and_phase(oracle_lib):
    """h~ = A f^(-7/6) exp(-i Psi): |h~| f^(7/6) is constant on the band and
    arg h~ = -Psi mod 2 pi; zero outside the band."""
    N, fs = 1 << 14, 4096.0
    h, (lo, hi) = oracle_lib.htilde(2.0, 3.0, N, fs, 40.0)
    k = np.arange(N // 2 + 1)
    f = k * fs / N
    amp = np.abs(h[lo:hi]) * f[lo:hi] ** (7.0 / 6.0)
    assert np.max(np.abs(amp / amp[0] - 1)) < 1e-12
    ph = oracle_lib.psi(2.0, 3.0, f[lo:hi])
    d = np.angle(h[lo:hi] * np.exp(1j * ph))
    assert np.max(np.abs(d)) < 1e-9
    assert np.all(h[:lo] == 0) and np.all(h[hi:] == 0)
    Mc = (6.0) ** 0.6 / 5.0 ** 0.2
    assert abs(amp[0] - Mc ** (5.0 / 6.0)) < 1e-12


def _quadrupole_chirp_spectrum(m1, m2, fs, Nfft, f_start, f_rise, f_fall, f_end):
    """Numerical Fourier transform of a Newtonian (quadrupole) inspiral in the
    time domain, built from the Peters-Mathews relations and not from any
    frequency-domain template formula: with tau = t_c - t and M_c in seconds,
      f(tau)   = (1/pi) (5 / (256 tau))^(3/8) M_c^(-5/8),
      Phi(tau) = -2 (tau / (5 M_c))^(5/8),
      h(t)     = M_c^(5/3) (pi f)^(2/3) cos Phi,
    the quadrupole amplitude up to a distance factor.  Cosine tapers in time
    switch the signal on between f_start and f_rise and off between f_fall and
    f_end.  Returns dt * rfft(h) on k = 0..Nfft/2."""
    M = m1 + m2
    mc = (m1 * m2 / M ** 2) ** 0.6 * M * _msun_s()

    def tau_of(f):
        return (5.0 / 256.0) * mc ** (-5.0 / 3.0) * (np.pi * f) ** (-8.0 / 3.0)

    dt = 1.0 / fs
    t0, t1, t2, t3 = tau_of(f_start), tau_of(f_rise), tau_of(f_fall), tau_of(f_end)
    assert t0 - t3 < Nfft * dt, "the chirp must fit the transform length"
    tau = t0 - np.arange(int((t0 - t3) / dt)) * dt
    f = (5.0 / (256.0 * tau)) ** 0.375 * mc ** (-0.625) / np.pi
    phi = -2.0 * (tau / (5.0 * mc)) ** 0.625
    h = mc ** (5.0 / 3.0) * (np.pi * f) ** (2.0 / 3.0) * np.cos(phi)
    w = np.ones_like(tau)
    on = tau > t1
    w[on] = 0.5 * (1.0 - np.cos(np.pi * (t0 - tau[on]) / (t0 - t1)))
    off = tau < t2
    w[off] = 0.5 * (1.0 + np.cos(np.pi * (t2 - tau[off]) / (t2 - t3)))
    return np.fft.rfft(h * w, Nfft) * dt


def _msun_s():
    return 4.925490947e-6   # G Msun / c^3 in seconds (IAU nominal)


def test_htilde_amplitude_is_stationary_phase_of_quadrupole_chirp(oracle_lib):
    """The Newtonian amplitude of the Sec. 1.1 templates, pinned without the
    oracle's formula: the FFT of a time-domain quadrupole chirp (amplitude
    M_c^(5/3) f^(2/3), Newtonian frequency sweep) divided by |h~| of the
    oracle must be one and the same constant at every in-band frequency and
    for every mass pair.  Stationary phase gives |h~(f)| = (A/2) fdot^(-1/2)
    with fdot = (96/5) pi^(8/3) M_c^(5/3) f^(11/3), so the constant is
    sqrt(5/384) pi^(-2/3) (G Msun/c^3)^(5/6) for the oracle's A = M_c^(5/6)
    in solar masses.  A wrong power of f or of M_c in h~ changes the ratio
    with frequency or between the two binaries (by 47 % for M_c^(5/3))."""
    fs, Nfft = 2048.0, 1 << 18
    f = np.arange(Nfft // 2 + 1) * fs / Nfft
    mid = (f >= 50.0) & (f <= 200.0)   # well inside the tapers; SPA corrections < 0.1 % here
    const = math.sqrt(5.0 / 384.0) * math.pi ** (-2.0 / 3.0) * _msun_s() ** (5.0 / 6.0)
    for m1, m2 in [(1.4, 1.4), (2.5, 2.0), (3.0, 1.2)]:
        H = _quadrupole_chirp_spectrum(m1, m2, fs, Nfft, 25.0, 35.0, 300.0, 400.0)
        h, _ = oracle_lib.htilde(m1, m2, Nfft, fs, 20.0)
        ratio = np.abs(H[mid]) / np.abs(h[mid])
        assert np.max(np.abs(ratio / const - 1.0)) < 3e-3, (m1, m2, ratio.min() / const, ratio.max() / const)


def test_mirror_symmetry(oracle_lib):
    """(m1, m2) and (m2, m1) are the same binary: identical template."""
    h1, b1 = oracle_lib.htilde(1.3, 2.7, 4096, 4096.0, 40.0)
    h2, b2 = oracle_lib.htilde(2.7, 1.3, 4096, 4096.0, 40.0)
    assert b1 == b2 and np.array_equal(h1, h2)


# ------------------------------------------------------- filter (Eq. 1) ----

def _correlate_time_domain(Hk, s, N, fs):
    """c_j = dt sum_n a_{(n+j) mod N} s_n, with a the real sequence whose
    one-sided spectrum is Hk (k = 0..N/2): a_n = df sum_k H_k e^{2 pi i nk/N}
    over the Hermitian extension.  Brute-force O(N^2) correlation."""
    dt = 1.0 / fs
    df = fs / N
    a = np.fft.irfft(Hk, n=N) * N * df
    c = np.empty(N)
    for j in range(N):
        c[j] = dt * np.dot(np.roll(a, -j), s)
    return c


def test_z_equals_time_domain_correlation(oracle_lib):
    """Eq. (1) against an independent time-domain circular correlation.

    x(t) = Re z is twice the correlation of s with the whitened template
    a_c (spectrum h~_c / S_n); with h~_c = -i h~_s (Sec. 1.1 quadrature
    relation) Im z is minus twice the correlation with a_s (spectrum
    h~_s / S_n = i h~_c / S_n)."""
    N, fs, f_low = 2048, 2048.0, 40.0
    rng = np.random.default_rng(11)
    s = rng.standard_normal(N)
    S = oracle_lib.psd_bins(N, fs)
    st = oracle_lib.data_spectrum(s, fs)
    m1, m2 = 4.0, 6.0
    out = oracle_lib.filter_template(m1, m2, st, S, N, fs, f_low)
    h, (lo, hi) = oracle_lib.htilde(m1, m2, N, fs, f_low)
    Hc = np.zeros(N // 2 + 1, dtype=complex)
    Hc[lo:hi] = h[lo:hi] / S[lo:hi]
    Hs = 1j * Hc
    cc = _correlate_time_domain(Hc, s, N, fs)
    cs = _correlate_time_domain(Hs, s, N, fs)
    scale = np.max(np.abs(out["z"]))
    assert np.max(np.abs(out["z"].real - 2 * cc)) < 1e-10 * scale
    assert np.max(np.abs(out["z"].imag + 2 * cs)) < 1e-10 * scale
    # and sigma^2 from Parseval on the whitened template: sigma^2 = 4 df sum |h|^2/S
    sig2 = 4 * fs / N * np.sum(np.abs(h[lo:hi]) ** 2 / S[lo:hi])
    assert abs(out["sigma"] ** 2 / sig2 - 1) < 1e-13
    assert np.max(np.abs(out["rho"] - np.abs(out["z"]) / out["sigma"])) < 1e-13 * np.max(out["rho"])


def test_quadrature_templates_orthogonal(oracle_lib):
    """h~_c = -i h~_s (Sec. 1.1): filtering the data r_c whose spectrum is
    the template itself gives z_0 = sigma^2 (Eq. 4), real and positive; the
    quadrature data r_s (spectrum i h~_c, orthogonal to r_c under the
    S_n-weighted inner product) gives z = -i z_c at every lag, so x and y swap
    roles and rho is the same series.  A conjugate on the wrong factor gives
    +i z_c; a filter that kept only x = Re z loses half of rho."""
    N, fs, f_low = 1 << 13, 2048.0, 40.0
    df = fs / N
    m1, m2 = 1.6, 2.3
    S = oracle_lib.psd_bins(N, fs)
    h, (lo, hi) = oracle_lib.htilde(m1, m2, N, fs, f_low)
    r_c = np.fft.irfft(h, n=N) * N * df
    r_s = np.fft.irfft(1j * h, n=N) * N * df
    # the two real signals are orthogonal in the whitened inner product
    # 4 Re sum a~ conj(b~)/S df, computed from their own DFTs
    a = np.fft.rfft(r_c) / fs
    b = np.fft.rfft(r_s) / fs
    ip = lambda u, v: 4 * df * np.real(np.sum(u[lo:hi] * np.conj(v[lo:hi]) / S[lo:hi]))
    assert abs(ip(a, b)) < 1e-12 * ip(a, a)
    assert abs(ip(b, b) / ip(a, a) - 1) < 1e-12
    zc = oracle_lib.filter_template(m1, m2, oracle_lib.data_spectrum(r_c, fs), S, N, fs, f_low)
    zs = oracle_lib.filter_template(m1, m2, oracle_lib.data_spectrum(r_s, fs), S, N, fs, f_low)
    sig2 = zc["sigma"] ** 2
    assert abs(zc["z"][0].real / sig2 - 1) < 1e-12
    assert abs(zc["z"][0].imag) < 1e-12 * sig2
    assert int(np.argmax(zc["rho"])) == 0 and abs(zc["rho"][0] - zc["sigma"]) < 1e-12 * zc["sigma"]
    scale = np.max(np.abs(zc["z"]))
    assert np.max(np.abs(zs["z"] + 1j * zc["z"])) < 1e-12 * scale
    assert np.max(np.abs(zs["rho"] - zc["rho"])) < 1e-12 * zc["sigma"]


def test_data_spectrum_is_scaled_dft(oracle_lib):
    N, fs = 512, 512.0
    s = np.random.default_rng(5).standard_normal(N)
    st = oracle_lib.data_spectrum(s, fs)
    ref = np.fft.rfft(s) / fs
    assert np.max(np.abs(st - ref)) < 1e-13


@pytest.mark.parametrize("N,fs,m", [(1 << 12, 4096.0, (1.4, 1.4)), (1 << 14, 4096.0, (2.0, 5.0)),
                                    (1 << 15, 2048.0, (1.3, 1.5))])
def test_noiseless_injection_recovers_snr_and_time(oracle_lib, N, fs, m):
    """An injection of the template itself, scaled to SNR and shifted by j0
    samples, peaks at rho = SNR exactly at j = (N - j0) mod N (literal Eq. 1
    with the conjugate on the data)."""
    rng = np.random.default_rng(N)
    for snr, j0 in [(10.0, int(rng.integers(0, N))), (7.5, 0), (20.0, N - 1)]:
        inj = np.zeros(1, dtype=oracle_lib.INJ_DTYPE)
        inj[0] = (m[0], m[1], snr, j0, rng.uniform(0, 2 * np.pi))
        s = oracle_lib.synth(np.zeros(2 * (N // 2)), N, fs, 40.0, inj)
        peaks, trig, n, _ = oracle_lib.filter_bank([m[0]], [m[1]], s, fs, 40.0, 6.0)
        assert abs(peaks["rho"][0] - snr) < 1e-9 * snr
        assert peaks["j"][0] == (N - j0) % N


def test_noise_statistics(oracle_lib):
    """Gaussian noise coloured by S_n: E[rho^2] = 2 and P(rho > r) = exp(-r^2/2)
    for the complex filter output (the optimal-statistic property, Sec. 1.1)."""
    N, fs = 1 << 16, 2048.0
    vals = []
    for seed in range(3):
        seg = workloads.SegmentSpec(N, fs, 900 + seed)
        s = oracle_lib.synth(seg.normals(), N, fs, 40.0)
        S = oracle_lib.psd_bins(N, fs)
        st = oracle_lib.data_spectrum(s, fs)
        out = oracle_lib.filter_template(1.4 + 0.1 * seed, 1.3, st, S, N, fs, 40.0)
        vals.append(out["rho"])
    rho = np.concatenate(vals)
    assert abs(np.mean(rho ** 2) - 2.0) < 0.06
    for r in (1.0, 2.0, 3.0):
        p = np.mean(rho > r)
        assert abs(p - math.exp(-r * r / 2)) < 0.1 * math.exp(-r * r / 2) + 2e-4


def test_noise_periodogram_matches_psd(oracle_lib):
    """The synthesised noise has one-sided PSD S_n: E|s~_k|^2 = T S_k / 2."""
    N, fs = 1 << 16, 2048.0
    seg = workloads.SegmentSpec(N, fs, 77)
    s = oracle_lib.synth(seg.normals(), N, fs, 40.0)
    st = np.fft.rfft(s) / fs
    S = oracle_lib.psd_bins(N, fs)
    T = N / fs
    k = np.arange(N // 2 + 1)
    band = (k >= 40 * 32) & (k < N // 2)
    ratio = np.abs(st[band]) ** 2 / (T * S[band] / 2)
    assert abs(np.mean(ratio) - 1.0) < 0.02
    assert np.all(np.abs(st[:40 * 32]) < 1e-12 * np.max(np.abs(st)))


def test_psd_scale_invariance(oracle_lib):
    """rho does not depend on the PSD scale S0 (physical 9e-46 vs whitened 1)."""
    N, fs = 1 << 13, 4096.0
    seg = workloads.SegmentSpec(N, fs, 5)
    inj = np.zeros(1, dtype=oracle_lib.INJ_DTYPE)
    inj[0] = (1.5, 1.5, 9.0, 1234, 0.3)
    g = seg.normals()
    a = oracle_lib.synth(g, N, fs, 40.0, inj, S0=1.0)
    b = oracle_lib.synth(g, N, fs, 40.0, inj, S0=9e-46)
    pa, *_ = oracle_lib.filter_bank([1.5, 2.0], [1.5, 1.1], a, fs, 40.0, 6.0, S0=1.0)
    pb, *_ = oracle_lib.filter_bank([1.5, 2.0], [1.5, 1.1], b, fs, 40.0, 6.0, S0=9e-46)
    assert np.max(np.abs(pa["rho"] - pb["rho"]) / pa["rho"]) < 1e-10
    assert np.array_equal(pa["j"], pb["j"])


def test_filter_bank_triggers_are_threshold_set(oracle_lib):
    """Triggers are exactly the samples with rho > thr, in (template, j) order;
    the peak is the first maximum."""
    N, fs = 1 << 12, 4096.0
    seg = workloads.SegmentSpec(N, fs, 8)
    inj = np.zeros(1, dtype=oracle_lib.INJ_DTYPE)
    inj[0] = (1.5, 1.6, 15.0, 100, 0.0)
    s = oracle_lib.synth(seg.normals(), N, fs, 40.0, inj)
    m1 = np.array([1.5, 1.4, 2.5])
    m2 = np.array([1.6, 1.7, 2.0])
    peaks, trig, n, _ = oracle_lib.filter_bank(m1, m2, s, fs, 40.0, 5.0)
    S = oracle_lib.psd_bins(N, fs)
    st = oracle_lib.data_spectrum(s, fs)
    expect = []
    for t in range(3):
        rho = oracle_lib.filter_template(m1[t], m2[t], st, S, N, fs, 40.0)["rho"]
        assert peaks["j"][t] == int(np.argmax(rho))
        expect += [(t, j) for j in np.nonzero(rho > 5.0)[0]]
    assert n == len(expect) > 0
    assert [(int(a), int(b)) for a, b in zip(trig["tmpl"], trig["j"])] == expect
    # capped output keeps the true count
    _, trig2, n2, _ = oracle_lib.filter_bank(m1, m2, s, fs, 40.0, 5.0, trig_cap=3)
    assert n2 == n and len(trig2) == 3


# ---------------------------------------------------------- refinement -----

def test_refine_objective_matches_filter_at_sample_times(oracle_lib):
    """The direct continuous-t sum equals rho^2 from the FFT path at t = j dt."""
    N, fs = 1 << 12, 4096.0
    seg = workloads.SegmentSpec(N, fs, 9)
    s = oracle_lib.synth(seg.normals(), N, fs, 40.0)
    S = oracle_lib.psd_bins(N, fs)
    st = oracle_lib.data_spectrum(s, fs)
    out = oracle_lib.filter_template(2.0, 1.5, st, S, N, fs, 40.0)
    for j in (0, 17, 2049, N - 1):
        J, _ = oracle_lib.refine_objective(2.0, 1.5, j / fs, st, S, N, fs, out["k_lo"], out["k_hi"])
        assert abs(J - out["rho"][j] ** 2) < 1e-10 * max(1.0, J)


def test_refine_gradient_matches_finite_differences(oracle_lib):
    """Analytic dJ/d(m1, m2, t) against FP64 central differences (h = 1e-6 Msun)."""
    N, fs = 1 << 14, 4096.0
    seg = workloads.SegmentSpec(N, fs, 10)
    inj = np.zeros(1, dtype=oracle_lib.INJ_DTYPE)
    inj[0] = (1.7, 1.3, 12.0, 3000, 0.4)
    s = oracle_lib.synth(seg.normals(), N, fs, 40.0, inj)
    S = oracle_lib.psd_bins(N, fs)
    st = oracle_lib.data_spectrum(s, fs)
    lo, hi = oracle_lib.band(N, fs, 40.0, oracle_lib.f_isco(1.72, 1.31))
    m1, m2 = 1.72, 1.31
    t = ((N - 3000) % N) / fs + 0.3 / fs
    J, g = oracle_lib.refine_objective(m1, m2, t, st, S, N, fs, lo, hi)
    hm, ht = 1e-6, 1e-7
    f = lambda a, b, c: oracle_lib.refine_objective(a, b, c, st, S, N, fs, lo, hi)[0]
    fd = np.array([(f(m1 + hm, m2, t) - f(m1 - hm, m2, t)) / (2 * hm),
                   (f(m1, m2 + hm, t) - f(m1, m2 - hm, t)) / (2 * hm),
                   (f(m1, m2, t + ht) - f(m1, m2, t - ht)) / (2 * ht)])
    for i in range(3):
        assert abs(g[i] - fd[i]) <= 1e-5 * max(abs(fd[i]), 1e-3 * np.max(np.abs(fd))), (i, g, fd)


def test_refine_stationary_at_true_parameters(oracle_lib):
    """Noiseless injection: J is maximal (= SNR^2) at the true (m1, m2, t), so
    the gradient vanishes there."""
    N, fs = 1 << 13, 4096.0
    inj = np.zeros(1, dtype=oracle_lib.INJ_DTYPE)
    inj[0] = (1.6, 1.4, 10.0, 500, 1.1)
    s = oracle_lib.synth(np.zeros(2 * (N // 2)), N, fs, 40.0, inj)
    S = oracle_lib.psd_bins(N, fs)
    st = oracle_lib.data_spectrum(s, fs)
    lo, hi = oracle_lib.band(N, fs, 40.0, oracle_lib.f_isco(1.6, 1.4))
    t = ((N - 500) % N) / fs
    J, g = oracle_lib.refine_objective(1.6, 1.4, t, st, S, N, fs, lo, hi)
    assert abs(J - 100.0) < 1e-8
    # scale of the gradient one sample or 0.01 Msun away
    _, g_off = oracle_lib.refine_objective(1.61, 1.4, t + 0.5 / fs, st, S, N, fs, lo, hi)
    assert np.all(np.abs(g) < 1e-6 * np.abs(g_off).max())


# ---------------------------------------------------------------------------
# Eq. (5), the chi^2 consistency test (Sec. 1.2)
# ---------------------------------------------------------------------------
def _chisq_case(oracle_lib, N, fs, seed, m=(1.5, 1.4), inj=None, noise_scale=1.0, p=16, edges=None):
    S = oracle_lib.psd_bins(N, fs)
    g = np.random.default_rng([seed, 77]).standard_normal(2 * (N // 2))
    s = oracle_lib.synth(g, N, fs, 40.0, inj, noise_scale=noise_scale)
    st = oracle_lib.data_spectrum(s, fs)
    return oracle_lib.chisq_series(m[0], m[1], st, S, N, fs, 40.0, p, edges=edges)


@pytest.mark.parametrize("p", [4, 16])
def test_chisq_noise_mean_is_2p_minus_2(oracle_lib, p):
    """In stationary Gaussian noise E[chi^2] = 2p - 2 for ANY partition of the
    band into p disjoint sub-bands: the bins are independent, so with
    E|z_l|^2 = 2 sigma_l^2 and no cross terms, (p/sigma^2) sum_l E|z_l - z/p|^2
    = (p/sigma^2)[2 sigma^2 (1 - 2/p) + 2 sigma^2 / p] = 2p - 2 (the paper's
    2p - 2 degrees of freedom).  Checked on the mean over 24 realisations."""
    means = [float(_chisq_case(oracle_lib, 1 << 13, 4096.0, seed, p=p)["chisq"].mean()) for seed in range(24)]
    m = float(np.mean(means))
    se = float(np.std(means, ddof=1) / np.sqrt(len(means)))
    assert se < 0.05 * (2 * p - 2)
    assert abs(m - (2 * p - 2)) < 4 * se + 1e-9, (m, se)


def test_chisq_single_band_is_zero(oracle_lib):
    r = _chisq_case(oracle_lib, 1 << 12, 4096.0, 3, p=1)
    assert np.max(np.abs(r["chisq"])) < 1e-20 * max(1.0, float(np.max(r["rho"]) ** 2)) + 1e-24


def test_chisq_band_edges_split_sigma2_equally(oracle_lib):
    """Edges run from k_lo to k_hi, increase, and each sub-band's sigma_l^2 is
    sigma^2/p to within one bin's |h|^2/S (the discretisation of the rule)."""
    N, fs, p = 1 << 14, 4096.0, 16
    r = _chisq_case(oracle_lib, N, fs, 5, p=p)
    h, (lo, hi) = oracle_lib.htilde(1.5, 1.4, N, fs, 40.0)
    S = oracle_lib.psd_bins(N, fs)
    q = np.abs(h[lo:hi]) ** 2 / S[lo:hi]
    e = r["edges"]
    assert e[0] == lo and e[-1] == hi and np.all(np.diff(e) > 0)
    df = fs / N
    sig2 = 4 * df * q.sum()
    assert np.isclose(r["sig2_l"].sum(), sig2, rtol=1e-12)
    assert np.max(np.abs(r["sig2_l"] - sig2 / p)) <= 4 * df * q.max() * (1 + 1e-9)


def test_chisq_matched_injection_closed_form(oracle_lib):
    """Noiseless data = the template itself at SNR rho0 coalescing at j0: at
    the peak z_l = conj(a) sigma_l^2 and z = conj(a) sigma^2 with |a| sigma =
    rho0, so chi^2 = p rho0^2 sum_l (sigma_l^2 - sigma^2/p)^2 / sigma^4."""
    N, fs, p = 1 << 14, 4096.0, 16
    inj = np.zeros(1, dtype=oracle_lib.INJ_DTYPE)
    inj[0] = (1.5, 1.4, 12.0, 3000, 0.7)
    r = _chisq_case(oracle_lib, N, fs, 1, inj=inj, noise_scale=0.0, p=p)
    jp = (N - 3000) % N
    assert int(np.argmax(r["rho"])) == jp and abs(r["rho"][jp] - 12.0) < 1e-9
    s2 = r["sig2_l"]
    sig2 = s2.sum()
    expect = p * 144.0 * np.sum((s2 - sig2 / p) ** 2) / sig2 ** 2
    assert abs(r["chisq"][jp] - expect) <= 1e-9 * max(expect, 1e-6)


def test_chisq_mismatched_signal_scales_with_snr_squared(oracle_lib):
    """A noiseless signal from another template: chi^2 is large at the peak and
    homogeneous of degree 2 in the signal amplitude (z_l and z scale by a)."""
    N, fs, p = 1 << 14, 4096.0, 16
    res = []
    for snr in (8.0, 16.0):
        inj = np.zeros(1, dtype=oracle_lib.INJ_DTYPE)
        inj[0] = (2.0, 1.1, snr, 2000, 0.0)
        res.append(_chisq_case(oracle_lib, N, fs, 2, m=(1.5, 1.4), inj=inj, noise_scale=0.0, p=p))
    j = int(np.argmax(res[1]["rho"]))
    assert res[1]["chisq"][j] > 2 * (2 * p - 2)           # far above the noise mean 2p - 2
    assert np.allclose(res[1]["chisq"], 4.0 * res[0]["chisq"], rtol=1e-9, atol=1e-12)


def test_chisq_given_edges_reproduce_rule(oracle_lib):
    r = _chisq_case(oracle_lib, 1 << 12, 4096.0, 9)
    r2 = _chisq_case(oracle_lib, 1 << 12, 4096.0, 9, edges=r["edges"])
    assert np.array_equal(r["chisq"], r2["chisq"])


# ---------------------------------------------------------------------------
# Trigger clustering (events)
# ---------------------------------------------------------------------------
def _random_triggers(oracle_lib, seed, n_t=5, n_seg=3, N=4000, per=60):
    rng = np.random.default_rng(seed)
    rows = []
    for t in range(n_t):
        for s in range(n_seg):
            js = np.unique(rng.integers(0, N, rng.integers(0, per)))
            for j in js:
                rows.append((t, s, int(j), 0, float(rng.choice([6.5, 7.0, 8.0, 9.5]) + rng.integers(0, 3)),
                             rng.standard_normal(), rng.standard_normal()))
    tr = np.array(rows, dtype=oracle_lib.TRIG_DTYPE) if rows else np.zeros(0, dtype=oracle_lib.TRIG_DTYPE)
    order = np.lexsort((tr["j"], tr["seg"], tr["tmpl"]))
    return tr[order]


def _brute_events(tr, W):
    """The same two-stage single linkage written as sorted runs in plain
    Python (stage 1: chains of triggers of one (tmpl, seg) at most W apart;
    stage 2: chains of the stage-1 winners of one segment)."""
    n = tr.size

    def comps(idx, key, group):
        idx = sorted(idx, key=key)
        groups, cur = [], []
        for i in idx:
            if cur and (group(i) != group(cur[-1]) or tr["j"][i] - tr["j"][cur[-1]] > W):
                groups.append(cur)
                cur = []
            cur.append(i)
        if cur:
            groups.append(cur)
        return groups

    g1 = comps(range(n), lambda i: (int(tr["tmpl"][i]), int(tr["seg"][i]), int(tr["j"][i])),
               lambda i: (int(tr["tmpl"][i]), int(tr["seg"][i])))
    win1 = []
    for g in g1:
        best = g[0]
        for i in g[1:]:
            if tr["rho"][i] > tr["rho"][best]:
                best = i
        win1.append((best, len(g)))
    cnt = {b: c for b, c in win1}
    g2 = comps([b for b, _ in win1], lambda i: (int(tr["seg"][i]), int(tr["j"][i]), int(tr["tmpl"][i])),
               lambda i: int(tr["seg"][i]))
    out = []
    for g in g2:
        best = g[0]
        for i in g[1:]:
            if tr["rho"][i] > tr["rho"][best]:
                best = i
        out.append((int(tr["tmpl"][best]), int(tr["seg"][best]), int(tr["j"][best]),
                    sum(cnt[i] for i in g), len(g), float(tr["rho"][best])))
    return out


@pytest.mark.parametrize("seed,W", [(1, 0), (2, 5), (3, 40), (4, 400), (5, 5000)])
def test_cluster_matches_python_runs(oracle_lib, seed, W):
    tr = _random_triggers(oracle_lib, seed)
    ev = oracle_lib.cluster(tr, W)
    ref = _brute_events(tr, W)
    got = [(int(e["tmpl"]), int(e["seg"]), int(e["j"]), int(e["n_trig"]), int(e["n_tmpl"]), float(e["rho"]))
           for e in ev]
    assert got == ref
    assert sum(e["n_trig"] for e in ev) == tr.size                # every trigger in exactly one event
    for a, b in zip(ev[:-1], ev[1:]):                             # sorted, separated events
        assert (a["seg"], a["j"]) < (b["seg"], b["j"])


def test_cluster_empty_and_single(oracle_lib):
    assert oracle_lib.cluster(np.zeros(0, dtype=oracle_lib.TRIG_DTYPE), 10).size == 0
    one = np.array([(3, 1, 77, 0, 6.2, 0.5, -0.5)], dtype=oracle_lib.TRIG_DTYPE)
    ev = oracle_lib.cluster(one, 10)
    assert ev.size == 1 and ev[0]["j"] == 77 and ev[0]["n_trig"] == 1 and ev[0]["n_tmpl"] == 1


# A trigger set worked by hand (window W = 10 samples).  Rows: (template,
# segment, j, rho).  Stage 1, per (template, segment), chains with gaps <= W:
#   t0 s0: {100, 105, 112} -> 105 (8.0, 3 triggers), {200} -> 200 (6.5)
#   t1 s0: {108} (9.0), {300} (6.1);  t2 s0: {118} (7.2), {129} (6.3), {210} (7.9)
#   t3 s0: {311} (6.0);  t0 s1: {100} (6.6)
#   s2: t0 {55}, t1 {55}, t3 {60}, all rho 7.0
# Stage 2, per segment in (j, template) order, chains with gaps <= W:
#   s0: 105 -3- 108 -10- 118 | 11 | 129 | 71 | 200 -10- 210 | 90 | 300 | 11 | 311
#   s2: 55 (t0) -0- 55 (t1) -5- 60: a three-way tie, kept by the lowest j, then template
HAND_TRIGGERS = [
    (0, 0, 100, 7.0), (0, 0, 105, 8.0), (0, 0, 112, 7.5), (0, 0, 200, 6.5),
    (1, 0, 108, 9.0), (1, 0, 300, 6.1),
    (2, 0, 118, 7.2), (2, 0, 129, 6.3), (2, 0, 210, 7.9),
    (3, 0, 311, 6.0),
    (0, 1, 100, 6.6),
    (3, 2, 60, 7.0), (1, 2, 55, 7.0), (0, 2, 55, 7.0),
]
# (template, segment, j, rho, n_trig, n_tmpl) of every event, in (segment, j) order
HAND_EVENTS = [
    (1, 0, 108, 9.0, 5, 3),
    (2, 0, 129, 6.3, 1, 1),
    (2, 0, 210, 7.9, 2, 2),
    (1, 0, 300, 6.1, 1, 1),
    (3, 0, 311, 6.0, 1, 1),
    (0, 1, 100, 6.6, 1, 1),
    (0, 2, 55, 7.0, 3, 3),
]


def test_cluster_hand_worked_set(oracle_lib):
    rows = [(t, s, j, 0, rho, 0.1 * j, -0.1 * t) for t, s, j, rho in HAND_TRIGGERS]
    tr = np.array(rows, dtype=oracle_lib.TRIG_DTYPE)
    tr = tr[np.lexsort((tr["j"], tr["seg"], tr["tmpl"]))]
    ev = oracle_lib.cluster(tr, 10)
    got = [(int(e["tmpl"]), int(e["seg"]), int(e["j"]), float(e["rho"]), int(e["n_trig"]), int(e["n_tmpl"]))
           for e in ev]
    assert got == HAND_EVENTS
    for e in ev:   # z travels with the loudest member
        assert e["z_re"] == 0.1 * e["j"] and e["z_im"] == -0.1 * e["tmpl"]
