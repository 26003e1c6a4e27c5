"""Seeded synthetic inputs for the signal-simulation hot path.

This module only draws numbers: ionization depositions ("depos": charge,
pitch position, drift time) and synthetic field/electronics responses.  It
holds none of the simulation arithmetic (no diffusion widths, no binning, no
transforms), so that both the CUDA path and the FP64 oracle can consume the
same inputs without sharing any of the method.

The paper's inputs are GEANT4 ionization groups (Sec. 2.2) and Wire-Cell
field responses (Sec. 2.1, the R term of Eq. 1); neither is available, so the
generators below stand in for them with the shapes and distributions of the
workloads the measurements use:

* ``uniform_depos``: depos uniform over the readout window, charge
  exponential (the single-plane deterministic workload).
* ``track_depos``: straight tracks sampled every ``step_mm``, charge per step
  Moyal distributed (a Landau-like shape), projected onto each wire plane's
  pitch axis (the three-plane, batched and large workloads).
* ``response``: a 2D response that is a Gaussian in wire times a
  Gaussian-derivative (bipolar, induction planes) or Gaussian (unipolar,
  collection plane) in time.
* ``noise_amplitudes``: amplitude spectra of the noise term of Eq. 1 (an
  electronics-shaped bump plus a white floor; a coherent bump shared by a
  group of channels).

All draws use ``numpy.random.Generator(PCG64(seed))``; every array is
contiguous float32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Detector constants of the workloads (mm, microseconds).
PITCH_MM = 5.0
TICK_US = 0.5
NTICKS = 6000
DRIFT_V_MM_US = 1.6
DL_MM2_US = 4.0e-4      # 4 cm^2/s
DT_MM2_US = 8.8e-4      # 8.8 cm^2/s
RESP_NWIRES = 21
RESP_NTICKS = 200
RESP_WIRE_CENTER = 10


@dataclasses.dataclass
class PlaneDepos:
    """Depos as seen by one wire plane (structure of arrays, float32)."""
    q: np.ndarray       # electrons
    x_mm: np.ndarray    # pitch coordinate from the low edge of wire 0
    t_us: np.ndarray    # drift time from the start of the readout window

    @property
    def n(self) -> int:
        return int(self.q.shape[0])

    def subset(self, idx) -> "PlaneDepos":
        return PlaneDepos(np.ascontiguousarray(self.q[idx]),
                          np.ascontiguousarray(self.x_mm[idx]),
                          np.ascontiguousarray(self.t_us[idx]))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def uniform_depos(n: int, nwires: int, seed: int, *, nticks: int = NTICKS,
                  pitch_mm: float = PITCH_MM, tick_us: float = TICK_US,
                  q_mean: float = 5000.0, t_min_us: float = 0.0) -> PlaneDepos:
    """Uniform pitch and drift time, exponential charge.

    Pitch ~ U[0, nwires*pitch), time ~ U(t_min, nticks*tick], charge ~
    Exp(q_mean).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(0.0, nwires * pitch_mm, n)
    t_max = nticks * tick_us
    # (0, t_max]: reflect the half-open uniform so that 0 is excluded.
    t = t_max - rng.uniform(0.0, t_max - t_min_us, n)
    q = rng.exponential(q_mean, n)
    return PlaneDepos(_f32(q), _f32(x), _f32(t))


@dataclasses.dataclass
class PlaneGeom:
    nwires: int
    angle_deg: float        # wire-pitch direction angle in the (y, z) plane
    bipolar: bool           # induction (bipolar) or collection (unipolar)


#: The three-plane detector: two induction planes at +-60 degrees, one
#: collection plane at 0 degrees.
THREE_PLANES = (PlaneGeom(800, 60.0, True), PlaneGeom(800, -60.0, True),
                PlaneGeom(960, 0.0, False))
#: The large three-plane detector of the precision study.
LARGE_PLANES = (PlaneGeom(2560, 60.0, True), PlaneGeom(2560, -60.0, True),
                PlaneGeom(3840, 0.0, False))


@dataclasses.dataclass
class TrackEvent:
    """Track depos of one event in 3D: drift coordinate, y, z and charge."""
    drift_mm: np.ndarray
    y_mm: np.ndarray
    z_mm: np.ndarray
    q: np.ndarray

    @property
    def n(self) -> int:
        return int(self.q.shape[0])

    def plane(self, geom: PlaneGeom, *, box_mm: float,
              drift_v: float = DRIFT_V_MM_US) -> PlaneDepos:
        """Project onto a plane's pitch axis (pitch = z cos a + y sin a).

        The pitch is shifted so that the centre of the transverse box lands
        on the centre of the plane's wire span; depos outside the span are
        kept (the simulation clips them bin by bin).
        """
        a = math.radians(geom.angle_deg)
        p = self.z_mm.astype(np.float64) * math.cos(a) + self.y_mm.astype(np.float64) * math.sin(a)
        centre = 0.5 * box_mm * (math.cos(a) + math.sin(a))
        p = p - centre + 0.5 * geom.nwires * PITCH_MM
        t = self.drift_mm.astype(np.float64) / drift_v
        return PlaneDepos(self.q.copy(), _f32(p), _f32(t))


def _reflect(v: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Fold coordinates into [lo, hi) by mirror reflection at the walls."""
    span = hi - lo
    u = np.mod(v - lo, 2.0 * span)
    u = np.where(u >= span, 2.0 * span - u, u)
    return np.clip(lo + u, lo, np.nextafter(hi, lo))


def track_event(n_depos: int, seed: int, *, steps_per_track: int = 500,
                step_mm: float = 1.0, box_mm: float = 2000.0,
                drift_len_mm: float = NTICKS * TICK_US * DRIFT_V_MM_US,
                q_mode: float = 6000.0, q_scale: float = 600.0,
                q_max: float = 60000.0) -> TrackEvent:
    """Straight tracks with isotropic directions, sampled every ``step_mm``.

    Start points are uniform in the transverse box [0, box)^2 and in the
    drift range [0, drift_len); the drift coordinate is folded back into the
    drift range by reflection so every depo has a valid drift time.  Charge
    per step is Moyal(mode, scale), drawn as mode - scale*ln(Z^2) with Z
    standard normal, clipped to [0, q_max].  The last track is truncated so
    exactly ``n_depos`` depos come out.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ntracks = max(1, -(-n_depos // steps_per_track))
    start = np.stack([rng.uniform(0.0, drift_len_mm, ntracks),
                      rng.uniform(0.0, box_mm, ntracks),
                      rng.uniform(0.0, box_mm, ntracks)], axis=1)
    cos_th = rng.uniform(-1.0, 1.0, ntracks)
    phi = rng.uniform(0.0, 2.0 * math.pi, ntracks)
    sin_th = np.sqrt(1.0 - cos_th * cos_th)
    direc = np.stack([cos_th, sin_th * np.cos(phi), sin_th * np.sin(phi)], axis=1)
    s = (np.arange(steps_per_track) + 0.5) * step_mm
    pts = start[:, None, :] + s[None, :, None] * direc[:, None, :]
    pts = pts.reshape(-1, 3)[:n_depos]
    z = rng.standard_normal(pts.shape[0])
    z = np.where(z == 0.0, 1e-300, z)
    q = np.clip(q_mode - q_scale * np.log(z * z), 0.0, q_max)
    drift = _reflect(pts[:, 0], 0.0, drift_len_mm)
    return TrackEvent(_f32(drift), _f32(pts[:, 1]), _f32(pts[:, 2]), _f32(q))


def event_depo_counts(nevents: int, seed: int, lo: int = 1000, hi: int = 500000) -> np.ndarray:
    """Per-event depo counts, log-uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), nevents))).astype(np.int64)


def response(kind: str = "bipolar", nwires: int = RESP_NWIRES, nticks: int = RESP_NTICKS,
             wire_center: int = RESP_WIRE_CENTER, wire_sigma: float = 1.5,
             tick_peak: float = 100.0, tick_sigma: float = 10.0) -> np.ndarray:
    """Synthetic response R[wire_offset + center][tick], float32, unit peak factors.

    Wire factor exp(-d^2 / (2 sw^2)); time factor -(u) exp(-u^2/2) (bipolar)
    or exp(-u^2/2) (unipolar) with u = (j - peak)/st.
    """
    d = np.arange(nwires, dtype=np.float64) - wire_center
    g = np.exp(-d * d / (2.0 * wire_sigma ** 2))
    u = (np.arange(nticks, dtype=np.float64) - tick_peak) / tick_sigma
    if kind == "bipolar":
        h = -u * np.exp(-0.5 * u * u)
    elif kind == "unipolar":
        h = np.exp(-0.5 * u * u)
    else:
        raise ValueError(f"unknown response kind {kind!r}")
    return _f32(np.outer(g, h))


def impact_response(kind: str = "bipolar", impacts: int = 10, nwires: int = RESP_NWIRES,
                    nticks: int = RESP_NTICKS, wire_center: int = RESP_WIRE_CENTER, wire_sigma: float = 1.5,
                    tick_peak: float = 100.0, tick_sigma: float = 10.0) -> np.ndarray:
    """Synthetic response at ``impacts`` positions inside the pitch,
    R[i][wire_offset + center][tick], float32: as ``response`` with the wire
    factor's centre moved to the charge's sub-pitch position,
    exp(-(d + 1/2 - (i + 1/2)/I)^2 / (2 sw^2)) (a charge near the pitch's low
    edge induces more on the lower neighbour)."""
    d = np.arange(nwires, dtype=np.float64) - wire_center
    u = (np.arange(nticks, dtype=np.float64) - tick_peak) / tick_sigma
    if kind == "bipolar":
        h = -u * np.exp(-0.5 * u * u)
    elif kind == "unipolar":
        h = np.exp(-0.5 * u * u)
    else:
        raise ValueError(f"unknown response kind {kind!r}")
    out = np.zeros((impacts, nwires, nticks))
    for i in range(impacts):
        shift = 0.5 - (i + 0.5) / impacts
        g = np.exp(-(d + shift) ** 2 / (2.0 * wire_sigma ** 2))
        out[i] = np.outer(g, h)
    return _f32(out)


def noise_amplitudes(L: int, kind: str = "incoherent", peak: float = 2.0e5, peak_frac: float = 0.1,
                     floor: float = 0.1) -> np.ndarray:
    """Synthetic noise amplitude spectrum on the L/2 + 1 half-spectrum bins of
    a length-L tick transform, float32: a shaped-electronics bump
    peak * (x / x0) * exp(1 - x / x0) over x = k / (L/2) (x0 = peak_frac of
    the Nyquist frequency) plus a white floor of floor * peak; the coherent
    kind is the same bump at 0.3x the height with no floor (it stands in
    for the noise a group of channels shares)."""
    k = np.arange(L // 2 + 1, dtype=np.float64)
    x = k / max(L / 2.0, 1.0)
    bump = (x / peak_frac) * np.exp(1.0 - x / peak_frac)
    if kind == "incoherent":
        return _f32(peak * (bump + floor))
    if kind == "coherent":
        return _f32(0.3 * peak * bump)
    raise ValueError(f"unknown noise kind {kind!r}")


# ---------------------------------------------------------------- workloads

@dataclasses.dataclass
class PlaneSpec:
    nwires: int
    nticks: int
    response: np.ndarray
    plane_id: int


@dataclasses.dataclass
class Workload:
    """One named workload: planes, per-event per-plane depos and parameters."""
    name: str
    planes: list            # list[PlaneSpec]
    events: list            # list[list[PlaneDepos]] indexed [event][plane]
    fluctuate: bool
    p_survive: float
    seed: int

    @property
    def n_depos(self) -> int:
        return sum(ev[0].n for ev in self.events)


def single_plane(n: int = 1000, seed: int = 1000, *, nwires: int = 960,
                 t_min_us: float = 0.0) -> Workload:
    """One plane of 960 wires x 6000 ticks, uniform depos, bipolar response,
    expected-value (no fluctuation) mode."""
    d = uniform_depos(n, nwires, seed, t_min_us=t_min_us)
    planes = [PlaneSpec(nwires, NTICKS, response("bipolar"), 0)]
    return Workload("single_plane_960x6000", planes, [[d]], False, 1.0, seed)


def three_planes(n: int = 100_000, seed: int = 1001, *, fluctuate: bool = True,
                 p_survive: float = 0.7) -> Workload:
    """Three planes 800/800/960 x 6000 with track depos and binomial fluctuation."""
    ev = track_event(n, seed)
    planes = [PlaneSpec(g.nwires, NTICKS, response("bipolar" if g.bipolar else "unipolar"), i)
              for i, g in enumerate(THREE_PLANES)]
    return Workload("three_planes_800_800_960x6000", planes,
                    [[ev.plane(g, box_mm=2000.0) for g in THREE_PLANES]],
                    fluctuate, p_survive, seed)


def three_planes_impacts(n: int = 100_000, seed: int = 1001, *, impacts: int = 10, fluctuate: bool = True,
                         p_survive: float = 0.7) -> Workload:
    """The three-plane event on planes whose response depends on the
    charge's position inside the pitch (``impacts`` sub-pitch positions,
    ``impact_response`` slices)."""
    w = three_planes(n, seed, fluctuate=fluctuate, p_survive=p_survive)
    planes = [PlaneSpec(sp.nwires, sp.nticks,
                        impact_response("bipolar" if g.bipolar else "unipolar", impacts=impacts), sp.plane_id)
              for sp, g in zip(w.planes, THREE_PLANES)]
    return Workload(f"three_planes_impacts{impacts}_800_800_960x6000", planes, w.events, fluctuate, p_survive, seed)


def batched_events(nevents: int = 64, seed: int = 1002, *, lo: int = 1000, hi: int = 500000,
                   fluctuate: bool = True, p_survive: float = 0.7) -> Workload:
    """Many events on the three-plane detector with log-uniform depo counts."""
    counts = event_depo_counts(nevents, seed, lo, hi)
    planes = [PlaneSpec(g.nwires, NTICKS, response("bipolar" if g.bipolar else "unipolar"), i)
              for i, g in enumerate(THREE_PLANES)]
    events = []
    for e, n in enumerate(counts):
        ev = track_event(int(n), seed + 1 + e)
        events.append([ev.plane(g, box_mm=2000.0) for g in THREE_PLANES])
    return Workload(f"batched_{nevents}ev_x3planes", planes, events, fluctuate, p_survive, seed)


def large_planes(n: int = 2_000_000, seed: int = 1004, *, fluctuate: bool = True,
                 p_survive: float = 0.7) -> Workload:
    """Three planes 2560/2560/3840 x 6000, 2,000 tracks of 1,000 steps."""
    ev = track_event(n, seed, steps_per_track=1000, box_mm=8000.0)
    planes = [PlaneSpec(g.nwires, NTICKS, response("bipolar" if g.bipolar else "unipolar"), i)
              for i, g in enumerate(LARGE_PLANES)]
    return Workload("large_2560_2560_3840x6000", planes,
                    [[ev.plane(g, box_mm=8000.0) for g in LARGE_PLANES]],
                    fluctuate, p_survive, seed)
