"""Learned warm start for a parametric family (the extension of Sec. 4.2's
warm start that the network of ``csrc/mlp.cu`` provides).

Pipeline, every arithmetic step in the library's kernels (this module only
moves device buffers and loops):
  1. solve training members with the family solver (``scs_family_*``) and
     keep each member's scaled state (u_x, u_y, v_s, u_tau) at its first
     passing test;
  2. standardise those targets per output (``scs_column_stats``,
     ``scs_standardize``);
  3. train the network theta -> standardised state with Adam on shuffled
     mini-batches (``scs_gather_rows``, ``scs_mlp_train_step``);
  4. for new members: network forward, prediction -> scaled warm start
     (``scs_warm_from_prediction``), y^ projected onto K* and s^ onto K
     (``scs_project``), then the warm-started solve.
The cold-started solve is the fallback: a warm start is only a starting
point, and the solver's own tests decide when a member is solved.

PyTorch only allocates device memory here.  Every library call of the
pipeline runs on one stream (the network's); it waits for PyTorch's copies
before using their buffers.
"""
from __future__ import annotations

import time

import numpy as np


class LearnedWarmStart:
    def __init__(self, fam, scs, torch, hidden=512, layers=3, batch=1024, seed=0, precision=1):
        self.fam, self.scs, self.torch = fam, scs, torch
        self.n = fam.A.shape[1]
        self.m = fam.A.shape[0]
        self.d_out = self.n + 2 * self.m + 1
        self.d_in = fam.d
        self.batch = batch
        self.precision = precision
        self.sizes = [self.d_in] + [hidden] * layers + [self.d_out]
        self.stream = torch.cuda.Stream()
        self.sp = self.stream.cuda_stream
        self.net = scs.MLP(self.d_in, hidden, layers, self.d_out, batch, stream=self.sp)
        rng = np.random.default_rng(seed)
        params = []
        for fin, fout in zip(self.sizes[:-1], self.sizes[1:]):
            params.append((rng.standard_normal((fout, fin)) / np.sqrt(fin), np.zeros(fout)))
        self.net.set_params(scs.pack_params(params))
        self.mean = torch.empty(self.d_out, device="cuda")
        self.sd = torch.empty(self.d_out, device="cuda")

    # ------------------------------------------------------------------ data
    def bc(self, thetas):
        pairs = [self.fam.bc(t) for t in thetas]
        return np.stack([b for b, _ in pairs]), np.stack([c for _, c in pairs])

    def solve_family(self, thetas, warm=None, chunk=16384):
        """Solve members in chunks; returns (infos, seconds, states) where
        states is a device tensor (count x d_out, float32) of the scaled
        states at the first passing test.  warm: optional callable
        (chunk thetas) -> (xh, yh, sh) device tensors (FP64, scaled)."""
        torch, scs = self.torch, self.scs
        infos, secs = [], 0.0
        states = torch.empty((len(thetas), self.d_out), dtype=torch.float32, device="cuda")
        fam = None
        for a in range(0, len(thetas), chunk):
            th = thetas[a:a + chunk]
            B, Cs = self.bc(th)
            if fam is None or fam.count != len(th):
                if fam is not None:
                    fam.close()
                fam = scs.Family(self.fam.A, self.fam.cone, B, Cs, precision=self.precision)
            else:
                fam.set_data(B, Cs)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if warm is not None:
                xh, yh, sh = warm(th)
                fam.warm_start_scaled_device(xh.data_ptr(), yh.data_ptr(), sh.data_ptr())
            infos += fam.solve_info()
            torch.cuda.synchronize()
            secs += time.perf_counter() - t0
            fam.snapshots(states[a:a + len(th)].data_ptr())
        if fam is not None:
            fam.close()
        torch.cuda.synchronize()
        return infos, secs, states

    # ------------------------------------------------------------- training
    def fit(self, thetas, states, epochs=30, lr=1e-3, seed=0, log_every=0):
        """Standardise the targets (in place) and train; returns the
        per-epoch mean loss (losses read back once per epoch)."""
        torch, scs = self.torch, self.scs
        N = states.shape[0]
        X = torch.tensor(np.asarray(thetas, dtype=np.float32), device="cuda")
        xb = torch.empty((self.batch, self.d_in), device="cuda")
        tb = torch.empty((self.batch, self.d_out), device="cuda")
        self.stream.wait_stream(torch.cuda.current_stream())
        scs.column_stats(states.data_ptr(), N, self.d_out, self.mean.data_ptr(), self.sd.data_ptr(), self.sp)
        scs.standardize(states.data_ptr(), N, self.d_out, self.mean.data_ptr(), self.sd.data_ptr(), self.sp)
        rng = np.random.default_rng(seed)
        steps_per_epoch = N // self.batch
        total = epochs * steps_per_epoch
        hist = []
        step = 0
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(N)[:steps_per_epoch * self.batch], dtype=torch.int64, device="cuda")
            self.stream.wait_stream(torch.cuda.current_stream())
            acc = 0.0
            for k in range(steps_per_epoch):
                idx = perm[k * self.batch:(k + 1) * self.batch]
                scs.gather_rows(X.data_ptr(), self.d_in, idx.data_ptr(), self.batch, xb.data_ptr(), self.sp)
                scs.gather_rows(states.data_ptr(), self.d_out, idx.data_ptr(), self.batch, tb.data_ptr(), self.sp)
                rate = lr * 0.5 * (1.0 + np.cos(np.pi * step / total))      # cosine decay
                want = k == steps_per_epoch - 1
                loss = self.net.train_step(xb.data_ptr(), tb.data_ptr(), rate, want_loss=want)
                if want:          # reading the loss synchronises the stream (perm may then be replaced)
                    acc = loss
                step += 1
            hist.append(acc)
            if log_every and (ep + 1) % log_every == 0:
                print(f"epoch {ep + 1}: loss {acc:.4f}", flush=True)
        return hist

    # ------------------------------------------------------------ inference
    def predict_warm(self, thetas, tau_min=1e-3):
        """Scaled warm starts (xh, yh, sh: FP64 device tensors) for members."""
        torch, scs = self.torch, self.scs
        cnt = len(thetas)
        nb = (cnt + self.batch - 1) // self.batch
        X = torch.zeros((nb * self.batch, self.d_in), device="cuda")
        X[:cnt] = torch.tensor(np.asarray(thetas, dtype=np.float32), device="cuda")
        P = torch.empty((nb * self.batch, self.d_out), device="cuda")
        xh = torch.empty((cnt, self.n), dtype=torch.float64, device="cuda")
        yh = torch.empty((cnt, self.m), dtype=torch.float64, device="cuda")
        sh = torch.empty((cnt, self.m), dtype=torch.float64, device="cuda")
        self.stream.wait_stream(torch.cuda.current_stream())
        for k in range(nb):
            self.net.forward(X[k * self.batch:].data_ptr(), P[k * self.batch:].data_ptr())
        scs.warm_from_prediction(P.data_ptr(), self.d_out, self.mean.data_ptr(), self.sd.data_ptr(), self.n, self.m,
                                 cnt, tau_min, xh.data_ptr(), yh.data_ptr(), sh.data_ptr(), self.sp)
        scs.project(self.fam.cone, 1, yh.data_ptr(), yh.data_ptr(), cnt, self.sp)
        scs.project(self.fam.cone, 0, sh.data_ptr(), sh.data_ptr(), cnt, self.sp)
        self.stream.synchronize()
        return xh, yh, sh

    def close(self):
        self.net.close()
