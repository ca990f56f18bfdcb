"""Time marching of slab problems with a learned Newton warm start (orchestration of C-ABI calls).

Sec. 3 of the paper marches the slab problems of Eq. (2.2) in time and solves
each one by a damped Newton method whose linear systems go to the GMRES-GMG
solver.  Every slab needs an initial guess: the fallback repeats the previous
slab's end value at every Radau node (stg_slab_initial_guess).  The warm start
(stg_warm_start) extrapolates linearly from the end values of the last two
slabs and adds the correction of a small convolutional network trained (on the
GPU, stg_cnn_train) on the slabs the march itself produced.  This module only
sequences library calls; all arithmetic runs in libstg.so.
"""
from __future__ import annotations

import time

import numpy as np

from . import Cnn, Solver


NEWTON_ATOL = 1e-8   # Sec. 4: Newton stops at an absolute residual below 1e-8,
GMRES_ATOL = 1e-9    # and every GMRES solve at an absolute residual below 1e-9


class March:
    """Slab-by-slab time march of one 2D problem (k, nu, tau fixed) with Dirichlet data g.

    Newton and GMRES use the absolute stopping criteria of Sec. 4, so every initial
    guess of a slab is solved to the same tolerance."""

    def __init__(self, spec, k, nu, tau, v0, g, **options):
        import torch

        options = dict(dict(gmres_rtol=0.0, gmres_atol=GMRES_ATOL), **options)
        self.torch = torch
        self.spec, self.k, self.nu, self.tau, self.v0 = spec, k, nu, tau, np.asarray(v0, dtype=np.float64)
        R = spec.dim * np.prod([2 * c + 1 for c in spec.n])
        self.R = int(R)
        w = np.tile(np.asarray(v0, dtype=np.float64), (k + 1, 1))
        self.solver = Solver(spec, k, nu, tau, torch.from_numpy(w.ravel()).cuda(), linearisation="newton",
                             **options)
        self.N = self.solver.sizes()[0]
        self.S = self.N // (k + 1) - self.R
        self.g = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float64).ravel()).cuda()
        # slab 0: the initial velocity at every node, pressure 0
        X0 = np.zeros((k + 1, self.R + self.S))
        X0[:, :self.R] = v0
        self.X = [torch.from_numpy(X0.ravel()).cuda()]
        self.stats = []

    def companion_solver(self, **options):
        """Another context of the same slab problem (e.g. the plain FP64 form, or a tighter GMRES
        tolerance) for evaluate(); it is re-linearised by every Newton step it takes."""
        options = dict(dict(gmres_rtol=0.0, gmres_atol=GMRES_ATOL), **options)
        w = np.tile(self.v0, (self.k + 1, 1))
        return Solver(self.spec, self.k, self.nu, self.tau, self.torch.from_numpy(w.ravel()).cuda(),
                      linearisation="newton", **options)

    def end_velocity(self, X):
        """View of the nodal velocities at the last Radau node (t_n) of a slab vector."""
        off = self.k * (self.R + self.S)
        return X[off:off + self.R]

    def initial_residual(self, n, X0):
        """||F_{n+1}(X0)|| for slab n+1 starting from slab n (no Newton step is taken)."""
        _, _, _, res, _ = self.solver.newton_slab(X0, v_prev=self.end_velocity(self.X[n]), g=self.g, maxit=0)
        return res

    def solve_slab(self, n, X0, rtol=0.0, atol=NEWTON_ATOL, maxit=20, solver=None):
        """Slab n+1 from slab n and initial guess X0: (X, steps, GMRES its, ||F||, ok, seconds)."""
        solver = self.solver if solver is None else solver
        self.torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, steps, its, res, ok = solver.newton_slab(X0, v_prev=self.end_velocity(self.X[n]), g=self.g,
                                                    rtol=rtol, atol=atol, maxit=maxit)
        self.torch.cuda.synchronize()
        return X, steps, its, res, ok, time.perf_counter() - t0

    def run(self, n_slabs, atol=NEWTON_ATOL):
        """Marches slabs len(X) .. n_slabs with the fallback guess; keeps every slab vector."""
        while len(self.X) <= n_slabs:
            n = len(self.X) - 1
            X0 = self.solver.slab_initial_guess(self.X[n])
            r0 = self.initial_residual(n, X0)
            X, steps, its, res, ok, sec = self.solve_slab(n, X0, atol=atol)
            if not ok:
                raise RuntimeError(f"slab {n + 1}: Newton did not converge (||F|| = {res:.3e})")
            self.X.append(X)
            self.stats.append(dict(slab=n + 1, r0=r0, steps=steps, its=its, res=res, sec=sec))

    # -- learned warm start
    # The velocity increment dv = v_n - v_{n-1} of each slab sets that slab's scale_d: inputs and
    # targets are measured in units of the slab's own increment, so the network sees the same
    # distribution while the flow's rate of change decays or grows.
    def scale_d(self, n):
        return max(self.solver.warm_scales(self.X[n], self.X[n - 1])[1], 1e-30)

    def scale_v(self, slabs):
        """Root mean square of v_n over the slabs n."""
        sv = sum(self.solver.warm_scales(self.X[n], self.X[n - 1])[0] ** 2 for n in slabs)
        return float(np.sqrt(sv / len(slabs)))

    def training_set(self, slabs, sv):
        """Inputs/targets predicting slab n+1 from slabs n-1, n for n in `slabs` (float32 device)."""
        torch = self.torch
        H, W = self.solver.node_grid()
        d = self.spec.dim
        x = torch.empty((len(slabs), 2 * d, H, W), dtype=torch.float32, device="cuda")
        t = torch.empty((len(slabs), d * (self.k + 1), H, W), dtype=torch.float32, device="cuda")
        for i, n in enumerate(slabs):
            sd = self.scale_d(n)
            self.solver.warm_features(self.X[n], self.X[n - 1], sv, sd, out=x[i])
            self.solver.warm_target(self.X[n], self.X[n - 1], self.X[n + 1], sd, out=t[i])
        return x, t

    def train(self, channels, params0, slabs, epochs=100, batch=16, lr=2e-3, seed=0):
        """Trains a network on slabs n -> n+1 for n in `slabs`; returns (net, scale_v, losses, seconds)."""
        sv = self.scale_v(slabs)
        x, t = self.training_set(slabs, sv)
        H, W = self.solver.node_grid()
        net = Cnn(channels, H, W, max_batch=batch)
        net.set_params(params0)
        rng = np.random.default_rng(seed)
        steps_per_epoch = len(slabs) // batch
        order = np.concatenate([rng.permutation(len(slabs))[:steps_per_epoch * batch] for _ in range(epochs)])
        self.torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = net.train(x, t, order, batch, lr)
        self.torch.cuda.synchronize()
        return net, sv, losses, time.perf_counter() - t0

    def evaluate(self, slabs, net, sv, maxit=20, atol=NEWTON_ATOL, solver=None,
                 names=("fallback", "linear", "network")):
        """Solves slab n+1 for n in `slabs` from the fallback guess, the linear extrapolation and
        the network's guess (those of `names`), all to the same absolute Newton tolerance.  The
        solves run on `solver` (default: the march's own), e.g. a context of the same problem in
        another precision form or with a tighter GMRES tolerance; the guesses are the same."""
        out = {name: [] for name in names}
        for n in slabs:
            sd = self.scale_d(n)
            make = {"fallback": lambda: self.solver.slab_initial_guess(self.X[n]),
                    "linear": lambda: self.solver.warm_start(None, self.X[n], self.X[n - 1], sv, sd),
                    "network": lambda: self.solver.warm_start(net, self.X[n], self.X[n - 1], sv, sd)}
            for name in names:
                X0 = make[name]()
                r0 = self.initial_residual(n, X0)
                X, steps, its, res, ok, sec = self.solve_slab(n, X0, rtol=0.0, atol=atol, maxit=maxit, solver=solver)
                out[name].append(dict(slab=n + 1, r0=r0, tol=atol, steps=steps, its=its, res=res, ok=ok, sec=sec))
        return out

    # -- checkpoint / resume
    # Flat binary: 8-byte magic, int64 header [version, dim, n_x, n_y, k, N, slab n, n_params],
    # float64 [scale_v], float64 X_{n-1}, float64 X_n, float32 network parameters (n_params).
    MAGIC = b"STGMARCH"

    def save(self, path, net=None, scale_v=1.0):
        """Writes the last two slab vectors, the slab index and the network's parameters."""
        n = len(self.X) - 1
        if n < 1:
            raise ValueError("nothing to checkpoint before the first slab")
        params = net.get_params() if net is not None else np.zeros(0, np.float32)
        hdr = np.array([1, self.spec.dim, *self.spec.n[:2], self.k, self.N, n, params.size], dtype=np.int64)
        with open(path, "wb") as f:
            f.write(self.MAGIC)
            hdr.tofile(f)
            np.array([scale_v], dtype=np.float64).tofile(f)
            for X in (self.X[n - 1], self.X[n]):
                X.detach().cpu().numpy().astype(np.float64).tofile(f)
            params.astype(np.float32).tofile(f)

    def load(self, path):
        """Restores a checkpoint of the same problem; returns (slab index n, parameters, scale_v).
        The march continues with slab n + 1 exactly as the saved run would have."""
        with open(path, "rb") as f:
            if f.read(8) != self.MAGIC:
                raise ValueError(f"{path}: not a march checkpoint")
            hdr = np.fromfile(f, dtype=np.int64, count=8)
            version, dim, nx, ny, k, N, n, n_params = (int(v) for v in hdr)
            if version != 1 or (dim, nx, ny, k, N) != (self.spec.dim, *self.spec.n[:2], self.k, self.N):
                raise ValueError(f"{path}: checkpoint of another problem")
            scale_v = float(np.fromfile(f, dtype=np.float64, count=1)[0])
            Xm = np.fromfile(f, dtype=np.float64, count=N)
            Xn = np.fromfile(f, dtype=np.float64, count=N)
            params = np.fromfile(f, dtype=np.float32, count=n_params)
        self.X = [None] * (n - 1) + [self.torch.from_numpy(Xm).cuda(), self.torch.from_numpy(Xn).cuda()]
        self.stats = []
        return n, params, scale_v

    def close(self):
        self.solver.close()


def summary(rows):
    """Totals and means of a list of per-slab records."""
    steps = sum(r["steps"] for r in rows)
    its = sum(r["its"] for r in rows)
    return dict(slabs=len(rows), newton_steps=steps, gmres_iters=its, mean_newton=steps / max(len(rows), 1),
                mean_gmres_per_newton=its / max(steps, 1), seconds=sum(r["sec"] for r in rows),
                max_final_over_tol=max((r["res"] / r["tol"] for r in rows if "tol" in r), default=None),
                mean_r0=float(np.mean([r["r0"] for r in rows])) if rows else None,
                all_converged=all(r.get("ok", True) for r in rows))
