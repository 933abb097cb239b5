"""Seeded synthetic inputs for the phase-space Monte Carlo (shared by tests, bench and smoke).

This module holds only *inputs*: parent masses, daughter masses, event counts, seeds and
request mixes.  It contains none of the method's arithmetic (no kinematics, no RNG of the
method, no weights), so both the CUDA path and the CPU oracle may draw their inputs from it
without sharing any computation.

The decays follow the workloads of the Hydra paper's phase-space example (§4.2, Listing 4:
a parent of given mass decaying to N daughters of given masses) at the sizes of the
benchmark configurations:

* ``B_TO_JPSI_K_PI``  — 3-body decay, M=5.2795 GeV -> (3.0969, 0.4937, 0.1396) GeV, seed 42.
* ``sweep_masses(N)``  — M=10 GeV, N=2..10 daughters, massless or massive with masses
  drawn uniformly in [0, M/(2N)] by ``numpy.random.default_rng(1000+N)``.
* ``D0_DALITZ``       — 3-body decay M=1.865 GeV -> (0.4937, 0.1396, 0.4937) GeV with the
  two-Breit-Wigner matrix-element parameters of the integration workload.
* ``batch_requests``  — uneven request mix: N uniform in 2..8, M uniform in [1, 10] GeV,
  masses uniform in [0, M/(2N)], events log-uniform in [1e3, 1e7], seed = base + i.
* ``serve_stream``    — Poisson arrivals (mean rate 2000/s) mixing generate and
  integrate requests.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# --- 3-body decay of a B+ -> J/psi K+ pi- like parent (FP64 output, 1e5 events) -------------
B_TO_JPSI_K_PI = dict(M=5.2795, masses=(3.0969, 0.4937, 0.1396), nevents=100_000, seed=42)

# --- N-body sweep ---------------------------------------------------------------------------
SWEEP_M = 10.0
SWEEP_N = tuple(range(2, 11))
SWEEP_NEVENTS = 100_000_000


def sweep_masses(n: int, massive: bool) -> tuple[float, ...]:
    """Daughter masses of the N-body sweep: zeros, or U[0, M/(2N)] from default_rng(1000+N)."""
    if not massive:
        return (0.0,) * n
    rng = np.random.default_rng(1000 + n)
    return tuple(float(v) for v in rng.uniform(0.0, SWEEP_M / (2 * n), size=n))


# --- D0 -> K pi K like Dalitz decay integrated against two Breit-Wigner amplitudes ----------
# params = (m0a, Gamma_a, m0b, Gamma_b, |c|, arg c); amplitude BW(s12; a) + c * BW(s23; b)
D0_DALITZ = dict(M=1.865, masses=(0.4937, 0.1396, 0.4937),
                 params=(0.892, 0.050, 1.020, 0.004, 0.5, 1.2),
                 nevents=1_000_000_000, seed=7)


# --- uneven batched requests ----------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Request:
    kind: str          # "generate" or "integrate"
    M: float
    masses: tuple
    nevents: int
    seed: int
    me: int = 0        # matrix-element id for integrate requests
    params: tuple = ()
    arrival: float = 0.0


def batch_requests(count: int = 4096, base_seed: int = 1_000_000, rng_seed: int = 20171115,
                   log_events: tuple[float, float] = (3.0, 7.0)) -> list[Request]:
    """Uneven generate requests: N~U{2..8}, M~U[1,10], m_i~U[0,M/(2N)], events log-uniform."""
    rng = np.random.default_rng(rng_seed)
    out = []
    for i in range(count):
        n = int(rng.integers(2, 9))
        M = float(rng.uniform(1.0, 10.0))
        masses = tuple(float(v) for v in rng.uniform(0.0, M / (2 * n), size=n))
        nev = int(round(10.0 ** rng.uniform(*log_events)))
        out.append(Request("generate", M, masses, nev, base_seed + i))
    return out


def serve_stream(rate_hz: float = 2000.0, duration_s: float = 30.0, rng_seed: int = 20171115,
                 gen_log_events: tuple[float, float] = (3.0, 6.0),
                 int_log_events: tuple[float, float] = (5.0, 8.0),
                 base_seed: int = 5_000_000) -> list[Request]:
    """Poisson request stream: half generate (N 2..8, float32 out), half Dalitz integrate."""
    rng = np.random.default_rng(rng_seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        if rng.random() < 0.5:
            n = int(rng.integers(2, 9))
            M = float(rng.uniform(1.0, 10.0))
            masses = tuple(float(v) for v in rng.uniform(0.0, M / (2 * n), size=n))
            nev = int(round(10.0 ** rng.uniform(*gen_log_events)))
            out.append(Request("generate", M, masses, nev, base_seed + i, arrival=t))
        else:
            nev = int(round(10.0 ** rng.uniform(*int_log_events)))
            out.append(Request("integrate", D0_DALITZ["M"], D0_DALITZ["masses"], nev,
                               base_seed + i, me=1, params=D0_DALITZ["params"], arrival=t))
        i += 1
    return out


def random_decay(rng: np.random.Generator, n: int, M: float | None = None,
                 massless_fraction: float = 0.2) -> tuple[float, tuple[float, ...]]:
    """A random decay (M, masses) for property tests: some daughters massless, the rest
    with masses up to M/(2N) so that the kinematic range is never empty."""
    if M is None:
        M = float(rng.uniform(0.5, 20.0))
    masses = rng.uniform(0.0, M / (2 * n), size=n)
    masses[rng.random(n) < massless_fraction] = 0.0
    return M, tuple(float(v) for v in masses)


def near_threshold_decay(n: int, M: float = 5.0, rel_gap: float = 1e-6) -> tuple[float, tuple]:
    """A decay whose kinetic energy T = M - sum(m) is a tiny fraction of M."""
    masses = np.full(n, M / n * (1.0 - rel_gap))
    return M, tuple(float(v) for v in masses)

