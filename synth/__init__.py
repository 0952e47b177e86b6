"""Seeded synthetic filterbank blocks.

Shared by the tests, the smoke check and the benchmark, and by nothing on the
product path.  It holds none of the search method's arithmetic: pulse arrival
offsets (the dispersion sweep) are always supplied by the caller, so this
module only draws noise, adds Gaussian pulse profiles at given per-channel
offsets, adds RFI shapes, and converts sample formats.

The workloads imitate the paper's: 1024 channels of 19.53 kHz between 398 and
418 MHz sampled every 51.2 us (Sec. 1.1), Gaussian noise, dispersed pulses of a
few ms, narrowband RFI occupying a few adjacent channels for a while and
broadband RFI occupying every channel for a sample (Sec. 2.2.1, Fig. 4).  The
paper's own data (telescope recordings and an undisclosed simulated file,
Sec. 3) are not available; these seeded blocks stand in for them.
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def noise(nchan, nsamp, seed, mean=0.0, std=1.0):
    """Gaussian noise, float32 (nchan, nsamp)."""
    g = rng(seed)
    x = g.standard_normal((nchan, nsamp), dtype=np.float32)
    if std != 1.0:
        x *= np.float32(std)
    if mean != 0.0:
        x += np.float32(mean)
    return x


def gaussian_profile(n, centre, fwhm):
    """Samples 0..n-1 of a unit-peak Gaussian with the given centre and FWHM."""
    s = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    t = np.arange(n, dtype=np.float64)
    return np.exp(-0.5 * ((t - centre) / s) ** 2)


def add_pulse(x, arrival, fwhm, amplitude):
    """Add amplitude * Gaussian(FWHM) centred at arrival[c] in every channel c.
    ``arrival`` is a per-channel sample offset supplied by the caller."""
    nchan, nsamp = x.shape
    s = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    half = int(np.ceil(6 * s)) + 1
    for c in range(nchan):
        a = float(arrival[c])
        lo = max(int(np.floor(a)) - half, 0)
        hi = min(int(np.ceil(a)) + half + 1, nsamp)
        if hi <= lo:
            continue
        t = np.arange(lo, hi, dtype=np.float64)
        x[c, lo:hi] += (amplitude * np.exp(-0.5 * ((t - a) / s) ** 2)).astype(x.dtype)
    return x


def add_narrowband(x, channels, t_lo, t_hi, level):
    """Narrowband RFI: raise the given channels by ``level`` over [t_lo, t_hi)."""
    for c in channels:
        x[c, t_lo:t_hi] += np.float32(level)
    return x


def add_broadband(x, times, level):
    """Broadband RFI: raise every channel by ``level`` at each given sample."""
    for t in times:
        x[:, t] += np.float32(level)
    return x


def poisson_bursts(nchan, nsamp, seed, rate_per_sample=1.0 / 32768, max_chans=16,
                   dur=(32, 2048), level=(5.0, 20.0)):
    """Random narrowband bursts: Poisson count, 1..max_chans adjacent channels,
    durations and levels uniform in the given ranges.  Returns a list of
    (c0, nch, t0, t1, level)."""
    g = rng(seed)
    n = g.poisson(rate_per_sample * nsamp)
    out = []
    for _ in range(n):
        nch = int(g.integers(1, max_chans + 1))
        c0 = int(g.integers(0, max(nchan - nch, 0) + 1))
        d = int(g.integers(dur[0], dur[1] + 1))
        t0 = int(g.integers(0, max(nsamp - d, 0) + 1))
        lv = float(g.uniform(level[0], level[1]))
        out.append((c0, nch, t0, t0 + d, lv))
    return out


def apply_bursts(x, bursts, scale=1.0):
    for c0, nch, t0, t1, lv in bursts:
        x[c0:c0 + nch, t0:t1] += np.float32(lv * scale)
    return x


def to_u8(x_float):
    """Round to nearest and clip to [0, 255]."""
    return np.clip(np.rint(x_float), 0, 255).astype(np.uint8)


def to_f16(x_float):
    return x_float.astype(np.float16)


def to_bf16_bits(x_float):
    """bfloat16 bit patterns (uint16), round to nearest even from float32."""
    b = np.ascontiguousarray(x_float, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) >> 16).astype(np.uint16)


def bf16_bits_to_f32(h):
    return (h.astype(np.uint32) << 16).view(np.float32)


# complex voltage samples of the beamformer output (Sec. 1.1: 16 bits for each
# complex component): int16 real part, then int16 imaginary part
C16 = np.dtype([("re", "<i2"), ("im", "<i2")])


def complex_voltage(envelope, seed, sigma=20.0):
    """Complex int16 voltages shaped like ``envelope`` (nchan, nsamp): each
    component is N(0, 1) * sigma * sqrt(envelope), rounded and clipped to
    int16, so the expected power follows the envelope (a pulse or an RFI
    burst drawn into the envelope raises the voltage variance there)."""
    g = rng(seed)
    amp = np.sqrt(np.maximum(np.asarray(envelope, np.float32), np.float32(0.0)))
    amp *= np.float32(sigma)
    out = np.empty(amp.shape + (2,), np.int16)
    v = np.empty(amp.shape, np.float32)
    for k in range(2):  # real, then imaginary part
        g.standard_normal(amp.shape, dtype=np.float32, out=v)
        v *= amp
        np.rint(v, out=v)
        np.clip(v, -32768, 32767, out=v)
        out[..., k] = v
    return out.view(C16)[..., 0]


# ---- workload recipes --------------------------------------------------------------
# Band of the paper's receiver (Sec. 1.1): 1024 channels over 398-418 MHz, 51.2 us.
BAND_1024 = dict(nchan=1024, f_lo=398.0, bw=20.0, t_samp=51.2e-6)


def single_block_workload(arrival_fn, seed=1000, nchan=1024, nsamp=32768, t0=12000,
                          snr=20.0, fwhm_ms=1.0, t_samp=51.2e-6, rfi_channels=(300, 301, 700, 701),
                          rfi_span=(8192, 12288), rfi_level=10.0, spikes=(5000, 20000, 26000),
                          spike_level=4.0):
    """One FP32 block: N(0,1) noise, one Gaussian pulse whose per-channel
    arrival is ``arrival_fn()`` + t0 (caller-supplied sweep), peak dedispersed
    SNR ``snr`` (per-channel peak snr / sqrt(nchan)), narrowband RFI on a few
    channels and broadband spikes."""
    x = noise(nchan, nsamp, seed)
    arr = np.asarray(arrival_fn(), dtype=np.float64) + t0
    add_pulse(x, arr, fwhm_ms * 1e-3 / t_samp, snr / np.sqrt(nchan))
    if rfi_channels:
        add_narrowband(x, rfi_channels, rfi_span[0], rfi_span[1], rfi_level)
    if spikes:
        add_broadband(x, spikes, spike_level)
    return x


# ---- device-side generation for large workloads ---------------------------------------
# Blocks of the wide-band and batched benchmark workloads are generated on the
# GPU with torch (noise from a seeded torch generator, pulses at caller-given
# per-channel arrivals, narrowband bursts) so that a 4096 x 2^18 block takes
# milliseconds instead of the host's tens of seconds.  No step of the method
# is computed here.

def torch_block(nchan, nsamp, seed, arrivals=(), rfi_channels=(), rfi_level=6.0, device="cuda",
                fmt="f32", u8_mean=128.0, u8_std=16.0):
    """One (nchan, nsamp) block on ``device``: N(0, 1) noise; for each
    (arrival[c], fwhm_samples, amplitude) in ``arrivals`` a Gaussian pulse
    centred at arrival[c] in channel c; for each channel in ``rfi_channels``
    a burst of +rfi_level over a random span of 10-50 % of the block.  The
    result in the storage format ``fmt``: "f32", "f16", "bf16" (int16 bit
    patterns, round to nearest even) or "u8" (round(x * u8_std + u8_mean)
    clipped to [0, 255])."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = torch.randn((nchan, nsamp), generator=g, device=device, dtype=torch.float32)
    for arr, fwhm, amp in arrivals:
        s = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
        half = int(np.ceil(6 * s)) + 1
        a = torch.as_tensor(np.asarray(arr, np.float64), device=device)
        base = torch.floor(a).to(torch.int64)
        k = torch.arange(-half, half + 2, device=device, dtype=torch.int64)
        t = base[:, None] + k[None, :]
        ok = (t >= 0) & (t < nsamp)
        prof = (amp * torch.exp(-0.5 * ((t.to(torch.float64) - a[:, None]) / s) ** 2)).to(torch.float32)
        rows = torch.arange(nchan, device=device)[:, None].expand_as(t)
        x.index_put_((rows[ok], t[ok]), prof[ok], accumulate=True)
    h = rng(int(seed) + 1)
    for c in rfi_channels:
        d = int(h.integers(nsamp // 10, nsamp // 2 + 1))
        t0 = int(h.integers(0, nsamp - d + 1))
        x[int(c), t0:t0 + d] += float(rfi_level)
    if fmt == "f32":
        return x
    if fmt == "f16":
        return x.to(torch.float16)
    if fmt == "bf16":
        return x.to(torch.bfloat16).view(torch.int16)
    if fmt == "u8":
        return torch.clamp(torch.round(x * u8_std + u8_mean), 0, 255).to(torch.uint8)
    raise ValueError(fmt)
