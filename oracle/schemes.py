"""The four FFT iteration schemes, step by step, in complex FP64.  Test
infrastructure only.

Problem (Eq. J12, J13): find E in U+E and J in U+J with J = sigma E,
sigma(x) = 1 + (sigma_1 - 1) chi(x); the effective conductivity follows from
Gamma_0 J = sigma_* Gamma_0 E.  Every scheme below reports, for its current
iterate, <E>, <J>, sigma_k = (<J>.e)/(<E>.e) (Eq. J13 projected on the applied
field e) and the mean squared field <|E|^2>.

Moulinec-Suquet, "ms" (Eq. J0-0 with sigma_0 of Eq. J1):
    E^{k+1} = e - Gamma_1[(sigma/sigma_0 - 1) E^k],   E^0 = e.

Eyre-Milton, "em" (reference sqrt(sigma_1), Eq. J2; the paper cites the scheme
without printing it, so the update below is derived from Eq. J12/J13): with
P = J + sigma_0 E and W = (sigma - sigma_0)/(sigma + sigma_0) pointwise one has
W P = J - sigma_0 E and (I - 2 Gamma_1) W P = P - 2 sigma_0 e, hence
    P^{k+1} = (I - 2 Gamma_1)(W P^k) + 2 sigma_0 e,   P^0 = (sigma + sigma_0) e,
    E = (P - W P)/(2 sigma_0),  J = (P + W P)/2.

Both schemes in the substituted space H'' (Eq. J27-J45), fields (Q, S, T) with S
and T zero in phase 2, local operator L'' = (t - 1) chi'' + I with
chi'' = (p p^T) chi (x) I_d (Eq. J36, J37), projection Gamma_1''(Q, S, T) =
(Gamma_1 Q, S, 0) (Eq. J44):
  "ms_sub" (Eq. J42a), reference (t + 1)/2:
    E''^{k+1} = e'' - Gamma_1''[(L''/sigma_0'' - 1) E''^k],  E''^0 = (e, 0, 0);
    the T component stays zero, so only (E_Q, S) are carried.
  "em_sub" (Eq. J43), reference sqrt(t); on phase 1 W'' = w (I - 2 p p^T) with
    w = (1 - sqrt t)/(1 + sqrt t), on phase 2 W'' = w on Q; the reflection
    I - 2 Gamma_1'' maps (Q, S, T) to ((I - 2 Gamma_1) Q, -S, T):
    P''^{k+1} = (I - 2 Gamma_1'')(W'' P''^k) + 2 sqrt(t) e'',
    P''^0 = (L'' + sqrt t) E''^0.
By Eq. J39-J42 the Q component of the converged E'' is the physical E and
sigma_* is unchanged.

Stop rule (the paper gives none; reading): r_k = |sigma_k - sigma_{k-1}|/|sigma_k|
and n_k = |<|E_k|^2> - <|E_{k-1}|^2>| / <|E_k|^2>; the iteration stops at the
first k with r_k < tol and n_k < tol for `consecutive` successive k (the field
must settle as well as sigma_*: the paper stresses that the fields are the
real interest, and a growing field component can leave sigma_* unchanged).
The update is then applied once more and the returned field, sigma_* and last
history entry belong to that final iterate.  A non-finite sigma_k or
<|E|^2>, or <|E|^2> above 1e12 times its first value, stops the run as
diverged (again after one more update); reaching max_iter updates without
convergence is "not converged".
"""
from __future__ import annotations

import cmath
from dataclasses import dataclass, field

import numpy as np

from . import constants as C
from .fourier import apply_gamma, fft, ifft

SCHEMES = ("ms", "em", "ms_sub", "em_sub")
STATUS_OK, STATUS_NOTCONV, STATUS_DIVERGED = 0, 3, 4
DIVERGENCE_FACTOR = 1e12


@dataclass
class Problem:
    mask: np.ndarray                 # uint8, shape (n_y, n_x) or (n_z, n_y, n_x)
    sigma1: complex
    e: np.ndarray                    # (d,) real applied field
    green: str = "trig"
    sigma_field: np.ndarray | None = None   # optional per-voxel sigma(x) (ms / em only)
    sigma0: complex | None = None            # reference medium for the per-voxel mode

    def __post_init__(self):
        self.mask = np.asarray(self.mask, dtype=np.uint8)
        self.e = np.asarray(self.e, dtype=np.float64)
        if self.e.shape != (self.mask.ndim,):
            raise ValueError("e must have d components")

    @property
    def d(self):
        return self.mask.ndim

    @property
    def shape(self):
        return self.mask.shape

    @property
    def chi(self):
        return self.mask.astype(np.float64)

    @property
    def sigma(self):
        if self.sigma_field is not None:
            return np.asarray(self.sigma_field, dtype=np.complex128)
        return 1.0 + (complex(self.sigma1) - 1.0) * self.chi

    def e_field(self):
        return np.broadcast_to(self.e.reshape((-1,) + (1,) * self.d), (self.d,) + self.shape).astype(np.complex128)


def _mean(f):
    d = f.ndim - 1
    return f.reshape(f.shape[0], -1).mean(axis=1) if d > 0 else f


def _set_mean(fhat, value_vec, N):
    """Put N * value at the zero frequency of every component."""
    idx = (slice(None),) + (0,) * (fhat.ndim - 1)
    fhat[idx] = N * np.asarray(value_vec)
    return fhat


class _Base:
    def __init__(self, pb: Problem):
        self.pb = pb
        self.N = int(np.prod(pb.shape))

    def observe(self, state):
        E, J = self.fields(state)
        mE, mJ = _mean(E), _mean(J)
        e = self.pb.e
        sig = complex(np.dot(mJ, e) / np.dot(mE, e))
        norm = float(np.mean(np.sum(np.abs(E) ** 2, axis=0)))
        return sig, mE, mJ, norm


class MS(_Base):
    """Moulinec-Suquet basic scheme (Eq. J0-0, J1)."""

    def __init__(self, pb: Problem):
        super().__init__(pb)
        if pb.sigma0 is not None:
            self.sigma0 = complex(pb.sigma0)
        elif pb.sigma_field is not None:
            s = np.asarray(pb.sigma_field).real
            self.sigma0 = complex((s.min() + s.max()) / 2.0)
        else:
            self.sigma0 = C.ms_sigma0(pb.sigma1)
        if self.sigma0 == 0:
            raise ValueError("reference medium sigma_0 = 0")

    def init_state(self):
        return {"Q": self.pb.e_field().copy()}

    def fields(self, st):
        E = st["Q"]
        return E, self.pb.sigma[None] * E

    def update(self, st):
        E = st["Q"]
        tau = (self.pb.sigma[None] / self.sigma0 - 1.0) * E
        Eh = -apply_gamma(fft(tau), self.pb.green)
        _set_mean(Eh, self.pb.e, self.N)
        return {"Q": ifft(Eh)}


class EM(_Base):
    """Eyre-Milton scheme with reference sqrt(sigma_1) (Eq. J2)."""

    def __init__(self, pb: Problem):
        super().__init__(pb)
        if pb.sigma0 is not None:
            self.sigma0 = complex(pb.sigma0)
        elif pb.sigma_field is not None:
            s = np.asarray(pb.sigma_field).real
            self.sigma0 = complex(np.sqrt(s.min() * s.max()))
        else:
            self.sigma0 = C.em_sigma0(pb.sigma1)
        if self.sigma0 == 0:
            raise ValueError("Eyre-Milton is undefined for sigma_0 = 0")
        s = self.pb.sigma
        self.W = (s - self.sigma0) / (s + self.sigma0)

    def init_state(self):
        return {"Q": (self.pb.sigma + self.sigma0)[None] * self.pb.e_field()}

    def fields(self, st):
        P = st["Q"]
        WP = self.W[None] * P
        return (P - WP) / (2.0 * self.sigma0), (P + WP) / 2.0

    def update(self, st):
        WP = self.W[None] * st["Q"]
        Wh = fft(WP)
        out = Wh - 2.0 * apply_gamma(Wh, self.pb.green)
        idx = (slice(None),) + (0,) * self.pb.d
        out[idx] += 2.0 * self.sigma0 * self.N * self.pb.e
        return {"Q": ifft(out)}


class MSSub(_Base):
    """Moulinec-Suquet applied in H'' (Eq. J36, J42a, J44)."""

    def __init__(self, pb: Problem, alpha: float, beta: float, sign2=1, sign3=1):
        super().__init__(pb)
        if pb.sigma_field is not None:
            raise ValueError("the substituted schemes need a two-phase medium")
        self.k = C.sub_constants(pb.sigma1, alpha, beta, sign2, sign3)
        self.s0 = (self.k.t + 1.0) / 2.0

    def init_state(self):
        z = np.zeros((self.pb.d,) + self.pb.shape, dtype=np.complex128)
        return {"Q": self.pb.e_field().copy(), "S": z}

    def _c(self, st):
        k = self.k
        return self.pb.chi[None] * (k.p1 * st["Q"] + k.p2 * st["S"])

    def fields(self, st):
        c = self._c(st)
        EQ = st["Q"]
        JQ = EQ + (self.k.t - 1.0) * self.k.p1 * c
        return EQ, JQ

    def update(self, st):
        k, s0, chi = self.k, self.s0, self.pb.chi[None]
        c = self._c(st)
        tauQ = ((k.t - 1.0) * k.p1 * c + (1.0 - s0) * st["Q"]) / s0
        tauS = chi * ((k.t - 1.0) * k.p2 * c + (1.0 - s0) * st["S"]) / s0
        Qh = -apply_gamma(fft(tauQ), self.pb.green)
        _set_mean(Qh, self.pb.e, self.N)
        return {"Q": ifft(Qh), "S": -tauS}

    def full_fields(self, st):
        """(E_Q, E_S, E_T) and (J_Q, J_S, J_T) of the current iterate."""
        k, chi = self.k, self.pb.chi[None]
        c = self._c(st)
        E = (st["Q"], st["S"], np.zeros_like(st["S"]))
        J = (E[0] + (k.t - 1.0) * k.p1 * c,
             E[1] + chi * (k.t - 1.0) * k.p2 * c,
             chi * (k.t - 1.0) * k.p3 * c)
        return E, J


class EMSub(_Base):
    """Eyre-Milton applied in H'' (Eq. J36, J43, J44)."""

    def __init__(self, pb: Problem, alpha: float, beta: float, sign2=1, sign3=1):
        super().__init__(pb)
        if pb.sigma_field is not None:
            raise ValueError("the substituted schemes need a two-phase medium")
        self.k = C.sub_constants(pb.sigma1, alpha, beta, sign2, sign3)
        self.rt = self.k.sqrt_t
        if self.rt == 0:
            raise ValueError("sqrt(t) = 0: sigma_1 = -alpha lies on the slit")
        self.w = (1.0 - self.rt) / (1.0 + self.rt)

    def init_state(self):
        k, chi, e = self.k, self.pb.chi[None], self.pb.e_field()
        c0 = chi * k.p1 * e                     # p . E''^0 on phase 1
        Q = (1.0 + self.rt) * e + (k.t - 1.0) * k.p1 * c0
        S = (k.t - 1.0) * k.p2 * c0
        T = (k.t - 1.0) * k.p3 * c0
        return {"Q": Q, "S": S, "T": T}

    def _WP(self, st):
        k, chi, w = self.k, self.pb.chi[None], self.w
        c = chi * (k.p1 * st["Q"] + k.p2 * st["S"] + k.p3 * st["T"])
        return (w * (st["Q"] - 2.0 * k.p1 * c),
                w * (st["S"] - 2.0 * k.p2 * c),
                w * (st["T"] - 2.0 * k.p3 * c))

    def fields(self, st):
        WQ, _, _ = self._WP(st)
        return (st["Q"] - WQ) / (2.0 * self.rt), (st["Q"] + WQ) / 2.0

    def update(self, st):
        WQ, WS, WT = self._WP(st)
        Wh = fft(WQ)
        out = Wh - 2.0 * apply_gamma(Wh, self.pb.green)
        idx = (slice(None),) + (0,) * self.pb.d
        out[idx] += 2.0 * self.rt * self.N * self.pb.e
        return {"Q": ifft(out), "S": -WS, "T": WT}

    def full_fields(self, st):
        WQ, WS, WT = self._WP(st)
        P = (st["Q"], st["S"], st["T"])
        W = (WQ, WS, WT)
        E = tuple((p - wp) / (2.0 * self.rt) for p, wp in zip(P, W))
        J = tuple((p + wp) / 2.0 for p, wp in zip(P, W))
        return E, J


def make_scheme(pb: Problem, scheme: str, alpha=None, beta=None, **kw):
    if scheme == "ms":
        return MS(pb)
    if scheme == "em":
        return EM(pb)
    if scheme == "ms_sub":
        return MSSub(pb, alpha, beta, **kw)
    if scheme == "em_sub":
        return EMSub(pb, alpha, beta, **kw)
    raise ValueError(f"unknown scheme {scheme!r}")


@dataclass
class Result:
    sigma_star: complex
    E: np.ndarray
    iterations: int
    status: int
    hist_sigma: np.ndarray
    hist_rel_change: np.ndarray
    hist_field_norm: np.ndarray
    mean_E: np.ndarray
    mean_J: np.ndarray
    state: dict = field(default_factory=dict)
    states: list = field(default_factory=list)


def solve(pb: Problem, scheme: str, alpha=None, beta=None, tol: float = 1e-10,
          max_iter: int = 1000, consecutive: int = 3, record_states: bool = False,
          **kw) -> Result:
    """Run one scheme with the stop rule described in the module docstring."""
    sch = make_scheme(pb, scheme, alpha, beta, **kw)
    st = sch.init_state()
    hs, hr, hn, states = [], [], [], []
    run = 0
    status = STATUS_NOTCONV
    norm0 = None
    for k in range(max_iter):
        if record_states:
            states.append({kk: v.copy() for kk, v in st.items()})
        sig, mE, mJ, norm = sch.observe(st)
        rel = abs(sig - hs[-1]) / abs(sig) if (k >= 1 and sig != 0) else np.inf
        nrel = abs(norm - hn[-1]) / norm if (k >= 1 and norm != 0) else np.inf
        hs.append(sig)
        hr.append(rel)
        hn.append(norm)
        if norm0 is None:
            norm0 = norm
        run = run + 1 if (rel < tol and nrel < tol) else 0
        diverged = (not np.isfinite(sig.real) or not np.isfinite(sig.imag) or not np.isfinite(norm)
                    or norm > DIVERGENCE_FACTOR * norm0)
        st = sch.update(st)
        if diverged:
            status = STATUS_DIVERGED
            break
        if run >= consecutive:
            status = STATUS_OK
            break
    iters = len(hs)
    if record_states:
        states.append({kk: v.copy() for kk, v in st.items()})
    sig, mE, mJ, norm = sch.observe(st)
    rel = abs(sig - hs[-1]) / abs(sig) if sig != 0 else np.inf
    hs.append(sig)
    hr.append(rel)
    hn.append(norm)
    E, _ = sch.fields(st)
    return Result(sig, E, iters, status, np.array(hs), np.array(hr), np.array(hn), mE, mJ, st, states)


def predicted_rate(scheme: str, sigma1: complex, alpha=None, beta=None, m_hull=None) -> float:
    """Asymptotic factor by which the error shrinks per iteration.

    em:     |z| with z = (sqrt(sigma_1) - 1)/(sqrt(sigma_1) + 1)   (Eq. J2)
    em_sub: |z| with z = (sqrt(t) - 1)/(sqrt(t) + 1)              (Eq. J4, J46)
            when [alpha, beta] contains every weighted pole.
    ms:     |z| max_n |1 - 2 m_n| with z = (sigma_1 - 1)/(sigma_1 + 1) (Eq. J1) and
            m_n the weighted eigenvalues of chi Gamma_1 chi (m_hull = (m_min, m_max)):
            the error operator is z Gamma_1 (1 - 2 chi).
    ms_sub: |(t - 1)/(t + 1)| (Eq. J42a) when [alpha, beta] contains every weighted pole.
    """
    if scheme == "em":
        return abs(C.em_z(sigma1))
    if scheme == "em_sub":
        t = C.t_of_sigma1(sigma1, alpha, beta)
        r = cmath.sqrt(t)
        return abs((r - 1) / (r + 1))
    if scheme == "ms":
        mmin, mmax = m_hull
        return abs(C.ms_z(sigma1)) * max(abs(1 - 2 * mmin), abs(1 - 2 * mmax))
    if scheme == "ms_sub":
        t = C.t_of_sigma1(sigma1, alpha, beta)
        return abs((t - 1) / (t + 1))
    raise ValueError(scheme)
