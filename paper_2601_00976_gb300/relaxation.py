"""Relaxation problem (Sec. 6.1): backward-Euler integration of the space-homogeneous
neutrino--matter system, one O(v/c) collision solve (collision_solve_v) per time step.

The paper's problem: rho = 1e12 g/cm^3, T = 7.6 MeV, Ye = 0.135 and v = (0.1, 0, 0) c; six
species with the same initial distribution
    f0(eps, mu) = 0.99 exp(-((eps - eps0) / sigma)^2 / 2) H(mu - mu0),
eps0 = 2 T, sigma = 10 MeV, mu0 = 0, whose angular moments are D = (1 - mu0) f_E / 2 and
I^1 = (1 - mu0^2) f_E / 4 with I^2 = I^3 = 0; Grid C (16 linear elements); dt from 1e-4 ms
growing by 1.04 per step up to 10 ms, until t = 100 ms; tol 1e-8, M_inner = M_outer = 2.

Each step is Algorithm 1 started from the previous step's state (backward Euler: the old
state is the previous solution, dtau = c dt).  Independent problems run as the nodes of one
call, so a batch of relaxation problems (other densities, temperatures, step schedules) costs
one launch per step.  This module only sequences calls and reads back observables; every
step runs in the library's kernels.
"""

import numpy as np

C_LIGHT = 2.99792458e10          # cm / s
M_B = 1.66053906660e-24          # g (the library's average baryon mass)
MEV_TO_ERG = 1.602176634e-6


def initial_moments(energies, ns, T, amplitude=0.99, sigma=10.0, mu0=0.0):
    """(D, I) of the paper's initial distribution at the node energies: shapes (ns, ne), (ns, ne, 3)."""
    e = np.asarray(energies, dtype=float)
    fE = amplitude * np.exp(-0.5 * ((e - 2.0 * T) / sigma) ** 2)
    D = np.broadcast_to(0.5 * (1.0 - mu0) * fE, (ns, e.size)).copy()
    I = np.zeros((ns, e.size, 3))
    I[:, :, 0] = 0.25 * (1.0 - mu0 * mu0) * fE
    return D, I


def schedule(dt0=1e-7, growth=1.04, dt_max=1e-2, t_end=0.1):
    """Time steps (s): dt0 growing by `growth` per step up to dt_max, the last one cut to end at t_end."""
    out, t, dt = [], 0.0, dt0
    while t < t_end * (1.0 - 1e-12):
        d = min(dt, dt_max, t_end - t)
        out.append(d)
        t += d
        dt *= growth
    return out


def rms_energy(D, energies, W3):
    """eps_RMS of Eq. rmsEnergy per node and species, sqrt(int D eps^5 / int D eps^3), by the energy
    quadrature: sqrt(sum_q W3 eps^2 D / sum_q W3 D)."""
    import torch
    e = torch.as_tensor(energies, dtype=D.dtype, device=D.device)
    w = torch.as_tensor(W3, dtype=D.dtype, device=D.device)
    return torch.sqrt(torch.sum(w * e * e * D, dim=-1) / torch.sum(w * D, dim=-1))


class Relaxation:
    """A batch of n independent relaxation problems on the GPU (CUDA float64 tensors).

    State: rho (n,), T (n,), Ye (n,), v (n, 3), D (n, ns, ne), I (n, ns, ne, 3).  `step(dt)`
    advances every problem by one backward-Euler step of length dt (scalar or (n,) seconds); the
    solve's outputs become the state, and two output sets alternate so that a call never writes
    the state it reads.  A zero-length step at construction fills in eps (the solve returns the
    inputs with their internal energy).
    """

    def __init__(self, ctx, params, rho, T, Ye, v, D, I, scale=None, freeze_velocity=False, v_floor=1e-6):
        import torch
        self.ctx, self.params = ctx, params
        self.rho, self.scale = rho, scale
        self.freeze, self.v_floor = freeze_velocity, v_floor
        n = rho.shape[0]
        f64 = dict(dtype=torch.float64, device=rho.device)
        i32 = dict(dtype=torch.int32, device=rho.device)

        def buffers():
            return dict(J=torch.empty_like(D), H=torch.empty_like(I), v=torch.empty_like(v),
                        Ye=torch.empty(n, **f64), eps=torch.empty(n, **f64), T=torch.empty(n, **f64),
                        n_outer=torch.empty(n, **i32), n_inner=torch.empty(n, **i32),
                        status=torch.empty(n, **i32))
        self._bufs = [buffers(), buffers()]
        self._k = 0
        self.state = dict(T=T.clone(), Ye=Ye.clone(), v=v.clone(), J=D.clone(), H=I.clone())
        self._dt = torch.empty(n, **f64)
        self.W2 = torch.tensor(ctx.w2, **f64)
        self.W3 = torch.tensor(ctx.w3, **f64)
        g = np.zeros(ctx.n_species)
        g[0] = 1.0
        if ctx.n_species > 1:
            g[1] = -1.0
        self.g = torch.tensor(g, **f64)
        self.t = 0.0
        self.steps = 0
        self.step(0.0)
        self.steps = 0

    def step(self, dt):
        s = self.state
        o = self._bufs[self._k % 2]
        if np.isscalar(dt):
            self._dt.fill_(dt)
        else:
            self._dt.copy_(dt)
        self.ctx.collision_solve_v(self.params, self.rho, s["T"], s["Ye"], s["v"], s["J"], s["H"], self._dt,
                                   self.scale, freeze_velocity=self.freeze, v_floor=self.v_floor, out=o)
        self.state = o
        self._k += 1
        self.t += float(dt) if np.isscalar(dt) else float(dt.max())
        self.steps += 1
        return o

    def totals(self):
        """Per problem: total lepton number density n_B Ye + N_nu (cm^-3) and total energy density
        rho eps_f + E_nu (erg/cm^3), with the Eulerian sums of Eqs. eulerianEnergyLG and
        eulerianNumberLG."""
        import torch
        s = self.state
        vI = torch.einsum("nsqi,ni->nsq", s["H"], s["v"])
        E = torch.einsum("q,nsq->n", self.W3, s["J"] + 2.0 * vI)
        N = torch.einsum("s,q,nsq->n", self.g, self.W2, s["J"] + vI)
        eps_f = s["eps"] + 0.5 * (s["v"] * s["v"]).sum(1) * C_LIGHT ** 2
        return self.rho * s["Ye"] / M_B + N, self.rho * eps_f + E * MEV_TO_ERG

    def rms(self):
        """eps_RMS per problem and species (Eq. rmsEnergy)."""
        return rms_energy(self.state["J"], self.ctx.energies, self.ctx.w3)

    def run(self, steps, record=None):
        """Advance through the time steps `steps`; record(self, k) is called after each step."""
        for k, dt in enumerate(steps):
            self.step(dt)
            if record is not None:
                record(self, k)
        return self
