"""The automatic Verlet update (Def. autoverlet) as a plain state machine.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Per-particle state is the reference position at the particle's last broad
phase and its skin, ``ref = (xref, yref, zref, skin)``.  Each step, given the
current positions (and velocities when the skin policy needs them):

1. flags  F = { p : |x_p - xref_p| > skin_p }           (Eq. update)
2. reference update, by trigger mode
   * ``TRIGGER_PARTIAL`` -- only p in F take xref_p = x_p and a fresh skin
     (the per-particle extension of the scheme; the pair set it yields is
     still correct by the triangle-inequality argument of Theorem 1,
     because every unflagged particle is within its skin of its own xref);
     with the early trigger (early_beta < 1), on a step where F is not
     empty, also every p with |x_p - xref_p| > early_beta * skin_p;
   * ``TRIGGER_GLOBAL``  -- if F is not empty every particle is updated: the
     paper's scheme, which re-executes the whole broad phase (Def.
     autoverlet);
   * ``TRIGGER_ALWAYS``  -- every particle every step: the broad phase
     "without Verlet buffer" that the paper compares against (Sec. Results).
3. pair set  P = { i < j : |xref_i - xref_j| <= R_NL,i + R_NL,j }
   (Def. verletlist / Eq. broad_phase), recomputed from scratch from the
   stored (xref, skin) -- it depends only on that state, not on history.
4. contacts  C = { (i, j) in P : delta_ij > 0 }            (Eq. delta)

The skin of a particle is fixed at its own update (reading: the paper's
K*v*dt rule uses the velocity of the step at which the list is built).
"""
from __future__ import annotations

import numpy as np

from . import (SKIN_GLOBAL, SKIN_DIAMETER_FACTOR, SKIN_PAPER_KVDT, SKIN_LEARNED,  # noqa: F401
               flags as _flags, flags_beta as _flags_beta, skin as _skin, pairs as _pairs,
               contacts as _contacts)

TRIGGER_PARTIAL, TRIGGER_GLOBAL, TRIGGER_ALWAYS = 0, 1, 2


class OracleLVB:
    """learned: for SKIN_LEARNED, a dict with "weights" (oracle.mlp.Weights)
    and "grid" (oracle.mlp.grid_params of the context); the proposal of each
    updated particle is then the network's, from the features of lvb_mlp.h."""

    def __init__(self, pos4, skin_kind, skin_value, dt, H, trigger=TRIGGER_PARTIAL,
                 vel4=None, proposal=None, ref4=None, learned=None, acc4=None,
                 early_beta=1.0):
        pos4 = np.ascontiguousarray(pos4, dtype=np.float32)
        self.n = len(pos4)
        self.kind, self.value, self.dt, self.H = int(skin_kind), np.float32(skin_value), \
            np.float32(dt), np.float32(H)
        self.trigger = int(trigger)
        # the early trigger (partial trigger only): on a step with a
        # violation, the particles past early_beta * skin are updated too
        self.early_beta = np.float32(early_beta)
        self.rad = pos4[:, 3].copy()
        self.learned = learned
        self.born = np.zeros(self.n, dtype=np.int64)
        if ref4 is not None:      # resume from a saved reference state
            self.ref = np.array(ref4, dtype=np.float32, copy=True)
        elif learned is not None:
            from . import mlp
            z = np.zeros(self.n, dtype=np.int64)
            f = mlp.features(pos4, vel4, acc4, dt, learned["grid"], np.zeros((self.n, 4), np.float32),
                             z, z, z)
            prop = mlp.infer(learned["weights"], f, (np.float32(2.0) * pos4[:, 3]))[0]
            self.ref = np.zeros((self.n, 4), dtype=np.float32)
            self.ref[:, :3] = pos4[:, :3]
            self.ref[:, 3] = _skin(SKIN_LEARNED, self.value, self.dt, self.H, pos4, vel4, prop)
        else:
            self.ref = np.zeros((self.n, 4), dtype=np.float32)
            self.ref[:, :3] = pos4[:, :3]
            self.ref[:, 3] = _skin(self.kind, self.value, self.dt, self.H, pos4, vel4, proposal)
        self.pi, self.pj = _pairs(self.ref, self.rad)
        self.steps = 0
        self.updates = 0          # particle reference updates (sum over steps of |U|)
        self.rebuild_steps = 0    # steps at which at least one reference changed

    def step(self, pos4, vel4=None, proposal=None, acc4=None):
        """Advance one step; returns (flags, updated) boolean arrays."""
        pos4 = np.ascontiguousarray(pos4, dtype=np.float32)
        f = _flags(pos4, self.ref)
        step = self.steps + 1
        if self.trigger == TRIGGER_PARTIAL:
            upd = f.copy()
            if self.early_beta < 1 and f.any():
                upd |= _flags_beta(pos4, self.ref, self.early_beta)
        elif self.trigger == TRIGGER_GLOBAL:
            upd = np.full(self.n, bool(f.any()))
        else:
            upd = np.ones(self.n, dtype=bool)
        if upd.any():
            idx = np.nonzero(upd)[0]
            v = None if vel4 is None else np.ascontiguousarray(vel4, dtype=np.float32)[idx]
            prop = None if proposal is None else np.asarray(proposal, dtype=np.float32)[idx]
            if self.learned is not None:
                prop = self._learned_proposal(idx, pos4, vel4, acc4, step)
            self.ref[idx, :3] = pos4[idx, :3]
            self.ref[idx, 3] = _skin(self.kind, self.value, self.dt, self.H, pos4[idx], v, prop)
            self.born[idx] = step
            self.pi, self.pj = _pairs(self.ref, self.rad)
            self.rebuild_steps += 1
            self.updates += len(idx)
        self.steps += 1
        return f, upd

    def contacts(self, pos4):
        return _contacts(self.pi, self.pj, pos4)

    def _learned_proposal(self, idx, pos4, vel4, acc4, step):
        """Network proposal from the state at the start of the step."""
        from . import mlp
        grid = self.learned["grid"]
        nrow = np.bincount(np.concatenate([self.pi, self.pj]), minlength=self.n)[idx]
        occ_all = np.bincount(mlp.cell_index(self.ref[:, :3], grid),
                              minlength=int(np.prod(grid["dims"])))
        occ = occ_all[mlp.cell_index(pos4[idx, :3], grid)]
        vel = np.asarray(vel4, np.float32)[idx]
        acc = np.asarray(acc4, np.float32)[idx]
        feats = mlp.features(pos4[idx], vel, acc, self.dt, grid, self.ref[idx], nrow,
                             step - self.born[idx], occ)
        self.last_features = (idx, feats)
        return mlp.infer(self.learned["weights"], feats, np.float32(2.0) * pos4[idx, 3])[0]


class RebuildLog:
    """The rebuild log (the skin network's training data, lvb_log_enable) as
    a plain procedure over an OracleLVB with the partial trigger.

    At every step, before the state machine updates anything:
      * the particles it is about to update (the flagged ones, Eq. update)
        that have no open record each open one: the step number, the
        position x_open, a running maximum m = 0, and the eight features of
        lvb_mlp.h from the state before the update (old reference state,
        partners in the current list, steps since the last update,
        reference positions in the cell of x);
    then the state machine steps; then, for every open record (including
    those just opened), m = max(m, |x - x_open|^2) at this step's position
    (binary32, fixed association), and a record opened `horizon` steps ago
    closes: it yields the sample (features, sqrt(m) / d) -- the largest
    displacement over the horizon in diameters -- and the particle may open
    a new record at a later update.

    grid: the cell grid of the features (oracle.mlp.grid_params)."""

    def __init__(self, sm, grid, horizon):
        if sm.trigger != TRIGGER_PARTIAL:
            raise ValueError("the rebuild log follows the partial trigger")
        self.sm, self.grid, self.horizon = sm, grid, int(horizon)
        n = sm.n
        self.t_open = np.full(n, -1, dtype=np.int64)
        self.x_open = np.zeros((n, 4), dtype=np.float32)
        self.m = np.zeros(n, dtype=np.float32)
        self.feat = np.zeros((n, 8), dtype=np.float32)
        self.samples = []

    def step(self, pos4, vel4=None, acc4=None, proposal=None):
        from . import mlp
        sm = self.sm
        pos4 = np.ascontiguousarray(pos4, dtype=np.float32)
        zero = np.zeros((sm.n, 4), dtype=np.float32)
        vel = zero if vel4 is None else np.asarray(vel4, dtype=np.float32)
        acc = zero if acc4 is None else np.asarray(acc4, dtype=np.float32)
        step = sm.steps + 1
        upd = _flags(pos4, sm.ref)
        idx = np.nonzero(upd & (self.t_open < 0))[0]
        if len(idx):
            nrow = np.bincount(np.concatenate([sm.pi, sm.pj]), minlength=sm.n)[idx]
            ncell = int(np.prod(self.grid["dims"]))
            occ_all = np.bincount(mlp.cell_index(sm.ref[:, :3], self.grid), minlength=ncell)
            occ = occ_all[mlp.cell_index(pos4[idx, :3], self.grid)]
            self.feat[idx] = mlp.features(pos4[idx], vel[idx], acc[idx], sm.dt, self.grid,
                                          sm.ref[idx], nrow, step - sm.born[idx], occ)
            self.t_open[idx] = step
            self.x_open[idx] = pos4[idx]
            self.m[idx] = np.float32(0)
        out = sm.step(pos4, vel4=vel4, proposal=proposal, acc4=acc4)
        o = np.nonzero(self.t_open >= 0)[0]
        if len(o):
            d = (pos4[o, :3] - self.x_open[o, :3]).astype(np.float32)
            d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]).astype(np.float32)
            d2 = (d2 + d[:, 2] * d[:, 2]).astype(np.float32)
            m = np.fmax(self.m[o], d2).astype(np.float32)
            close = (step - self.t_open[o]) >= self.horizon
            c = o[close]
            if len(c):
                diam = (np.float32(2.0) * sm.rad[c]).astype(np.float32)
                lab = (np.sqrt(m[close]).astype(np.float32) / diam).astype(np.float32)
                self.samples.append(np.concatenate([self.feat[c], lab[:, None]], axis=1))
                self.t_open[c] = -1
            self.m[o[~close]] = m[~close]
        return out

    def log(self):
        """The closed records so far, (k, 9) binary32, in closing order."""
        if not self.samples:
            return np.zeros((0, 9), dtype=np.float32)
        return np.concatenate(self.samples).astype(np.float32)
