"""Thin PyTorch-facing wrapper of the HOPE C ABI (include/hope.h).

PyTorch provides device memory and streams only; every step of the path runs in the
library's CUDA kernels.  Tensors must be contiguous CUDA tensors of the context's dtype
with hope_state_elems() elements (shape (3, 6, N, N) for one sphere).
"""
import ctypes

import numpy as np
import torch

from . import _lib as L

IC_GEOSTROPHIC, IC_ROSSBY, IC_DAMBREAK, IC_BUMPS = 2, 6, 7, 8
IC_MOUNTAIN_SURFACE, IC_MOUNTAIN_FLOW, IC_JET = 5, 10, 11
# section 5.4: umax, theta0, theta1, theta2, alpha, beta, hhat
JET = (80.0, 3.141592653589793 / 7, 5 * 3.141592653589793 / 14, 3.141592653589793 / 4, 1.0 / 3, 1.0 / 15, 120.0)
MOUNTAIN = (2000.0, 3.141592653589793 / 9, 1.5 * 3.141592653589793, 3.141592653589793 / 6)  # section 5.2
RADIUS, GRAVITY, OMEGA = 6.37122e6, 9.80616, 7.292e-5


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, ctx):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or t.dtype != ctx.dtype or t.numel() != ctx.elems:
        raise ValueError("expected a contiguous CUDA %s tensor of %d elements" % (ctx.dtype, ctx.elems))
    return ctypes.c_void_p(t.data_ptr())


class Sphere:
    """One HOPE context: a cubed sphere (or an ensemble of spheres) with its tables."""

    def __init__(self, N, order, scheme=L.HOPE_TPP, precision=L.HOPE_FP64, rk=L.HOPE_SSPRK3,
                 ghost_iters=10, radius=RADIUS, gravity=GRAVITY, omega=OMEGA, weno_eps=0.0,
                 coriolis_tilt=0.0):
        lib = L.load()
        p = L.default_params()
        p.radius, p.gravity, p.omega = radius, gravity, omega
        p.precision, p.rk, p.ghost_iters, p.weno_eps = precision, rk, ghost_iters, weno_eps
        p.coriolis_tilt = coriolis_tilt
        h = ctypes.c_void_p()
        if isinstance(N, (list, tuple)):
            arr = (ctypes.c_int * len(N))(*N)
            L.check(lib.hope_init_ensemble(len(N), arr, order, scheme, ctypes.byref(p), ctypes.byref(h)))
            self.members = list(N)
        else:
            L.check(lib.hope_init_grid(int(N), order, scheme, ctypes.byref(p), ctypes.byref(h)))
            self.members = [int(N)]
        self._h = h
        self.offsets = [0]
        for n in self.members:
            self.offsets.append(self.offsets[-1] + 18 * n * n)
        self.N = self.members[0]
        self.order, self.scheme, self.precision = order, scheme, precision
        self.radius, self.gravity, self.omega = radius, gravity, omega
        self.dtype = torch.float64 if precision == L.HOPE_FP64 else torch.float32
        self.elems = lib.hope_state_elems(h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().hope_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ state
    @property
    def shape(self):
        if len(self.members) == 1:
            return (3, 6, self.N, self.N)
        return (self.elems,)

    def member(self, q, m):
        """View of member m of an ensemble state as (3, 6, N_m, N_m)."""
        n = self.members[m]
        return q.view(-1)[self.offsets[m]:self.offsets[m + 1]].view(3, 6, n, n)

    def empty(self, device="cuda"):
        return torch.empty(self.shape, dtype=self.dtype, device=device)

    def initial_state(self, case, params, extra=None):
        q = self.empty()
        prm = (ctypes.c_double * len(params))(*params)
        ex = list(extra) if extra is not None else []
        exa = (ctypes.c_double * max(1, len(ex)))(*ex)
        L.check(L.load().hope_initial_state(self._h, case, prm, len(params), exa, len(ex),
                                            ctypes.c_void_p(q.data_ptr()), _stream()))
        return q

    def geostrophic(self, alpha=0.0, u0=None, phi0=2.94e4):
        if u0 is None:
            u0 = 2 * 3.141592653589793 * self.radius / (12 * 86400.0)
        return self.initial_state(IC_GEOSTROPHIC, [alpha, u0, phi0])

    def mountain_surface(self, hs0=MOUNTAIN[0], R=MOUNTAIN[1], lon_c=MOUNTAIN[2], lat_c=MOUNTAIN[3]):
        """Cell averages of sqrtG phi_s of the mountain of eq. 5.8, shape (6, N, N) on the
        device (pass to set_topography)."""
        return self.initial_state(IC_MOUNTAIN_SURFACE, [hs0, R, lon_c, lat_c])[0]

    def mountain_flow(self, alpha=0.0, u0=20.0, h0=5960.0, hs0=MOUNTAIN[0], R=MOUNTAIN[1],
                      lon_c=MOUNTAIN[2], lat_c=MOUNTAIN[3]):
        """Section 5.2's zonal flow over the mountain (depth state; h0 the free surface)."""
        return self.initial_state(IC_MOUNTAIN_FLOW, [alpha, u0, h0 * self.gravity, hs0, R, lon_c, lat_c])

    def galewsky(self, perturbed=True, phi0=0.0):
        """The perturbed jet of section 5.4; perturbed=False drops the bump of eq. 5.18;
        phi0 = 0 gives a mean depth of 10 km."""
        P = list(JET)
        if not perturbed:
            P[6] = 0.0
        return self.initial_state(IC_JET, P + [phi0])

    def rossby_haurwitz(self, w=7.848e-6, K=7.848e-6, R=4.0, h0=8000.0):
        return self.initial_state(IC_ROSSBY, [w, K, R, h0])

    def dam_break(self, lon=0.0, lat=0.0, radius=0.3490658503988659, h_in=10.0, h_out=1.0):
        return self.initial_state(IC_DAMBREAK, [lon, lat, radius, h_in, h_out])

    def bumps(self, centres, alpha=0.0, amp=50.0, radius=0.08726646259971647, u0=None, phi0=2.94e4):
        if u0 is None:
            u0 = 2 * 3.141592653589793 * self.radius / (12 * 86400.0)
        flat = [float(v) for c in centres for v in c]
        return self.initial_state(IC_BUMPS, [alpha, u0, phi0, amp, radius], flat)

    # ------------------------------------------------------------------ operator
    def tendency(self, q, out=None):
        if out is None:
            out = torch.empty_like(q)
        L.check(L.load().hope_tendency(self._h, _ptr(q, self), _ptr(out, self), _stream()))
        return out

    def step(self, q, dt, nsteps=1):
        """nsteps RK steps in place on q (a CUDA tensor)."""
        L.check(L.load().hope_step(self._h, _ptr(q, self), float(dt), int(nsteps), _stream()))
        return q

    def step_host(self, q_host, dt, nsteps=1, out=None):
        """End-to-end step on host memory (copies inside the call); returns out."""
        if q_host.is_cuda or not q_host.is_contiguous() or q_host.dtype != self.dtype:
            raise ValueError("expected a contiguous host tensor of the context dtype")
        if out is None:
            out = torch.empty_like(q_host)
        L.check(L.load().hope_step_host(self._h, ctypes.c_void_p(q_host.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), float(dt), int(nsteps), _stream()))
        return out

    def tendency_vjp(self, q, lam, out=None):
        """(dL/dq)^T lam at q (hand-written adjoint kernels)."""
        if out is None:
            out = torch.empty_like(q)
        L.check(L.load().hope_tendency_vjp(self._h, _ptr(q, self), _ptr(lam, self), _ptr(out, self), _stream()))
        return out

    def step_vjp(self, qn, lam_np1, dt, out=None):
        """(dS/dq)^T lam_np1 for one RK step S of size dt taken from qn."""
        if out is None:
            out = torch.empty_like(qn)
        L.check(L.load().hope_step_vjp(self._h, _ptr(qn, self), _ptr(lam_np1, self), _ptr(out, self), float(dt),
                                       _stream()))
        return out

    def step_ssprk3_vjp(self, qn, lam_np1, dt, out=None):
        """step_vjp of an SSP-RK3 step whatever the context's default stepper."""
        if out is None:
            out = torch.empty_like(qn)
        L.check(L.load().hope_step_ssprk3_vjp(self._h, _ptr(qn, self), _ptr(lam_np1, self), _ptr(out, self),
                                              float(dt), _stream()))
        return out

    def tape_bytes(self):
        """Bytes of one step's tape (stage states, ghost rings, edge points)."""
        n = ctypes.c_size_t()
        L.check(L.load().hope_tape_bytes(self._h, ctypes.byref(n)))
        return n.value

    def _tape_ptr(self, tape):
        if not tape.is_cuda or not tape.is_contiguous() or tape.dtype != torch.uint8 or \
                tape.numel() < self.tape_bytes():
            raise ValueError("expected a contiguous CUDA uint8 tensor of %d bytes" % self.tape_bytes())
        return ctypes.c_void_p(tape.data_ptr())

    def step_record(self, q, dt, tape):
        """One RK step of q in place, recording its tape (uint8 CUDA tensor)."""
        L.check(L.load().hope_step_record(self._h, _ptr(q, self), float(dt), self._tape_ptr(tape), _stream()))
        return q

    def step_vjp_tape(self, qn, tape, lam_np1, dt, out=None):
        """step_vjp for the step recorded in `tape` from qn, without forward recomputation."""
        if out is None:
            out = torch.empty_like(qn)
        L.check(L.load().hope_step_vjp_tape(self._h, _ptr(qn, self), self._tape_ptr(tape), _ptr(lam_np1, self),
                                            _ptr(out, self), float(dt), _stream()))
        return out

    def rollout(self, q0, dt, nsteps, checkpoint_every=10, tapes=True):
        """Differentiable nsteps-step integration: returns q(T) with a backward pass that
        recomputes each segment of `checkpoint_every` steps once from its checkpoint and
        applies the hand-written step adjoints in reverse.  With tapes=True the recompute
        records every step's tape (checkpoint_every x tape_bytes() of device memory) so
        the step adjoints run no forward work; with tapes=False each step adjoint
        recomputes its stages."""
        return _Rollout.apply(q0, self, float(dt), int(nsteps), int(checkpoint_every), bool(tapes))

    def mass(self, q):
        m = (ctypes.c_double * len(self.members))()
        L.check(L.load().hope_total_mass(self._h, _ptr(q, self), m, _stream()))
        return m[0] if len(self.members) == 1 else list(m)

    def status(self):
        s = ctypes.c_uint()
        L.check(L.load().hope_status(self._h, ctypes.byref(s)))
        return s.value

    def ghost_nnz(self):
        n, r = ctypes.c_longlong(), ctypes.c_longlong()
        L.check(L.load().hope_ghost_nnz(self._h, ctypes.byref(n), ctypes.byref(r)))
        return n.value, r.value

    def set_profiling(self, enable=True):
        L.check(L.load().hope_set_profiling(self._h, 1 if enable else 0))

    def kernel_times(self):
        """Per-kernel milliseconds of the most recent profiled step: a list of 3 stages x
        [ghost, reconstruction, flux, update]."""
        buf = (ctypes.c_float * 64)()
        n = ctypes.c_int()
        L.check(L.load().hope_kernel_times(self._h, buf, 64, ctypes.byref(n)))
        v = list(buf[:n.value])
        return [v[i:i + 4] for i in range(0, len(v), 4)]

    def vjp_phase_times(self):
        """Phases (ms) of the last persistent stage VJP of an ensemble, with profiling on:
        forward ghost, forward reconstruction, flux adjoint, reconstruction adjoint,
        gather, transposed ghost operator."""
        t = (ctypes.c_float * 6)()
        L.check(L.load().hope_vjp_phase_times(self._h, t))
        return list(t)

    def autotune(self, reps=5):
        """Re-time the tile shapes -- of the persistent stage (ensembles) or of the TPP
        reconstruction (one sphere) -- and keep the fastest; returns (per-candidate ms,
        (tx, ty), resident grid or tile count).  The times list has one entry per candidate
        (three for one sphere; the candidate list of the persistent stage for an ensemble)."""
        ms = (ctypes.c_float * L.HOPE_AUTOTUNE_MAX)()
        tx, ty, grid = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(L.load().hope_autotune(self._h, reps, ms, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(grid)))
        n = 3 if len(self.members) == 1 else L.load().hope_autotune_candidates(self._h)
        return list(ms)[:n], (tx.value, ty.value), grid.value

    def recon_tile(self):
        """(tx, ty): cells per block of the per-kernel TPP reconstruction."""
        tx, ty = ctypes.c_int(), ctypes.c_int()
        L.check(L.load().hope_recon_tile(self._h, ctypes.byref(tx), ctypes.byref(ty)))
        return tx.value, ty.value

    def set_recon_tile(self, tx, ty):
        L.check(L.load().hope_set_recon_tile(self._h, int(tx), int(ty)))

    def set_topography(self, phis_avg):
        """Bottom topography: cell averages of sqrtG * phi_s, shape (6, N, N) (any array
        convertible to FP64 on the host); None removes it."""
        if phis_avg is None:
            L.check(L.load().hope_set_topography(self._h, None))
            return
        if hasattr(phis_avg, "detach"):
            phis_avg = phis_avg.detach().cpu().numpy()
        a = np.ascontiguousarray(np.asarray(phis_avg, dtype=np.float64))
        if a.shape != (6, self.N, self.N):
            raise ValueError("topography must have shape (6, N, N)")
        L.check(L.load().hope_set_topography(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def launches_per_stage(self):
        n = ctypes.c_int()
        L.check(L.load().hope_launches_per_stage(self._h, ctypes.byref(n)))
        return n.value


def measure_fma_peak(precision):
    r = ctypes.c_double()
    L.check(L.load().hope_measure_fma_peak(precision, ctypes.byref(r)))
    return r.value


def measure_fma_peak_clock(precision, reps=8):
    """(flops/s, SM MHz during the measured launch, flops per SM per clock cycle)."""
    r, mhz, fpc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    L.check(L.load().hope_measure_fma_peak_clock(precision, reps, ctypes.byref(r), ctypes.byref(mhz),
                                                 ctypes.byref(fpc)))
    return r.value, mhz.value, fpc.value


class _Rollout(torch.autograd.Function):
    """q(T) = S^n(q0) with checkpointed recompute and hand-written step adjoints."""

    @staticmethod
    def forward(ctx, q0, sphere, dt, nsteps, every, tapes):
        work = q0.detach().clone().contiguous()
        ckpts = [work.clone()]
        for s in range(nsteps):
            sphere.step(work, dt)
            if (s + 1) % every == 0 and s + 1 < nsteps:
                ckpts.append(work.clone())
        ctx.sphere, ctx.dt, ctx.nsteps, ctx.every, ctx.ckpts, ctx.tapes = sphere, dt, nsteps, every, ckpts, tapes
        return work

    @staticmethod
    def backward(ctx, lam):
        sphere, dt, nsteps, every = ctx.sphere, ctx.dt, ctx.nsteps, ctx.every
        lam = lam.detach().contiguous().clone()
        work = torch.empty_like(lam)
        buf = torch.empty_like(lam)
        tb = (sphere.tape_bytes() + 255) // 256 * 256 if ctx.tapes else 0  # rows 256-B aligned
        tape = torch.empty((min(every, nsteps), tb), dtype=torch.uint8, device=lam.device) if ctx.tapes else None
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * every
            n = min(every, nsteps - start)
            work.copy_(ctx.ckpts[seg])
            states = [work.clone()]
            for k in range(n - 1 if tape is None else n):
                if tape is None:
                    sphere.step(work, dt)
                else:
                    sphere.step_record(work, dt, tape[k])
                if k < n - 1:
                    states.append(work.clone())
            for s in reversed(range(n)):
                if tape is None:
                    sphere.step_vjp(states[s], lam, dt, out=buf)
                else:
                    sphere.step_vjp_tape(states[s], tape[s], lam, dt, out=buf)
                lam, buf = buf, lam
        ctx.ckpts = None
        return lam, None, None, None, None, None
