"""Sharding the method across ranks on CPU (gloo, world size 2), with the compute on host cores.

(a) Instances split by cost across two ranks: the union of the ranks' results equals the
    single-process run bitwise (each instance is evaluated by the same code either way).
(b) One evaluation split by source and by target: each rank forms the type-1 Fourier coefficients
    of its source shard (the paper's discrete formula, Section 5.2 eqs. disrete_sigma_hat and
    sh_fourier, summed here with numpy), the ranks all-reduce them, and each rank evaluates its
    target shard.  Linearity in the sources makes the sum exact; the result is checked against the
    oracle's discrete formula and its direct sum at the plan tolerance.
"""
import math
import os
import socket

import numpy as np
import pytest

import oracle
import oracle.params as OP
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instances():
    rng = np.random.default_rng(21)
    out = []
    for _ in range(9):
        n = int(rng.integers(200, 900))
        out.append(W.random_instance(rng, n, float(np.exp(rng.uniform(np.log(3.0), np.log(60.0))))))
    return out


def _instance_result(wk):
    delta = OP.delta_from_mesh(wk.alpha, wk.h_vol)
    return oracle.direct_sum(wk.alpha, delta, wk.xs, wk.ys, wk.q, wk.xt, wk.yt)


class _Problem:
    """A small single-layer + volume problem and the discrete formula's parameters for it."""

    def __init__(self):
        rng = np.random.default_rng(4)
        self.alpha, self.delta, self.tol = 10.0, 0.0167, 1e-10
        n_s, n_t = 300, 160
        self.xs, self.ys = rng.uniform(-1.0, 1.0, n_s), rng.uniform(-1.0, 1.0, n_s)
        self.q = rng.normal(size=n_s) / n_s
        self.xt, self.yt = rng.uniform(-1.0, 1.0, n_t), rng.uniform(-1.0, 1.0, n_t)
        eps = self.tol / 4
        kmax = OP.kmax_relative(self.alpha, self.delta, eps)
        self.period = 2.0 + OP.r_tol(self.alpha, self.delta, eps)
        self.M = OP.modes(kmax, self.period)
        self.center = (0.0, 0.0)
        m = np.arange(-self.M, self.M + 1)
        dk = 2 * math.pi / self.period
        self.kx, self.ky = np.meshgrid(dk * m, dk * m, indexing="ij")
        s = self.alpha ** 2 + self.kx ** 2 + self.ky ** 2
        self.mult = np.exp(-self.delta * s) / s / self.period ** 2

    def coefficients(self, lo, hi):
        """F(m) = sum_j q_j exp(-i k_m . y_j) over sources [lo, hi), as (re, im) planes."""
        ph = (np.multiply.outer(self.kx, self.xs[lo:hi] - self.center[0]) +
              np.multiply.outer(self.ky, self.ys[lo:hi] - self.center[1]))
        F = (np.exp(-1j * ph) * self.q[lo:hi]).sum(axis=-1)
        return np.stack([F.real, F.imag])

    def finish(self, F, lo, hi):
        """u(x_i) = Re sum_m mult(m) F(m) exp(i k_m . x_i) for targets [lo, hi)."""
        Fc = (F[0] + 1j * F[1]) * self.mult
        ph = (np.multiply.outer(self.kx, self.xt[lo:hi] - self.center[0]) +
              np.multiply.outer(self.ky, self.yt[lo:hi] - self.center[1]))
        return (np.exp(1j * ph) * Fc[..., None]).sum(axis=(0, 1)).real


def _rank_main(rank, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2606_28865_b300 import sharding
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    works = _instances()
    res = sharding.evaluate_instances([wk.n_src * wk.n_trg for wk in works],
                                      lambda i: _instance_result(works[i]), dist)
    np.savez(os.path.join(out_dir, f"inst{rank}.npz"), **{str(i): v for i, v in res.items()})
    pb = _Problem()
    u = sharding.evaluate_source_sharded(
        len(pb.xs), len(pb.xt), lambda lo, hi: torch.from_numpy(pb.coefficients(lo, hi)),
        lambda F, lo, hi: pb.finish(F.numpy(), lo, hi), dist)
    np.save(os.path.join(out_dir, f"src{rank}.npy"), u)
    dist.destroy_process_group()


def test_split_helpers():
    from paper_2606_28865_b300 import sharding
    assert [sharding.split_range(10, 3, r) for r in range(3)] == [(0, 4), (4, 7), (7, 10)]
    assert sharding.split_range(1, 2, 1) == (1, 1)
    parts = sharding.assign_instances([5, 1, 4, 2, 3], 2)
    assert sorted(parts[0] + parts[1]) == [0, 1, 2, 3, 4]
    loads = [sum([5, 1, 4, 2, 3][i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= 1


def test_two_gloo_ranks_shard_instances_and_one_evaluation(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    # (a) both ranks hold every instance's result, bitwise equal to the one-process run
    works = _instances()
    for r in range(2):
        got = np.load(tmp_path / f"inst{r}.npz")
        assert sorted(int(k) for k in got.files) == list(range(len(works)))
        for i, wk in enumerate(works):
            assert np.array_equal(got[str(i)], _instance_result(wk)), (r, i)
    # (b) the source-sharded evaluation against the oracle
    pb = _Problem()
    u0, u1 = np.load(tmp_path / "src0.npy"), np.load(tmp_path / "src1.npy")
    assert np.array_equal(u0, u1)
    disc = oracle.discrete_sum(pb.alpha, pb.delta, pb.period, pb.M, pb.center, pb.xs, pb.ys,
                               pb.q, pb.xt, pb.yt)
    direct = oracle.direct_sum(pb.alpha, pb.delta, pb.xs, pb.ys, pb.q, pb.xt, pb.yt)
    scale = np.max(np.abs(direct))
    assert np.max(np.abs(u0 - disc)) <= 1e-13 * np.abs(pb.q).sum() * 10
    assert np.max(np.abs(u0 - direct)) <= pb.tol * scale
