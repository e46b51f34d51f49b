"""Host-side helpers of bench.py (no GPU): the null-space route's keywords and the table of ncu
DRAM traffic that the roofline objects quote."""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


class _Problem:
    def __init__(self, ncoil, kernel, rank):
        self.ncoil, self.kernel, self.rank = ncoil, kernel, rank


def test_eig_kwargs_default_route_adds_nothing():
    assert bench.eig_kwargs(argparse.Namespace(eig_solver="tridiag"), _Problem(8, (5, 5, 1), 75)) == {}
    assert bench.eig_kwargs(argparse.Namespace(), _Problem(8, (5, 5, 1), 75)) == {}


def test_eig_kwargs_rsvd_test_vectors():
    args = argparse.Namespace(eig_solver="rsvd")
    # l = r + max(r/2, 8), at most n = C k^d
    assert bench.eig_kwargs(args, _Problem(32, (5, 5, 1), 45)) == {"eig_solver": "rsvd", "rsvd_cols": 67,
                                                                    "rsvd_seed": 23}
    assert bench.eig_kwargs(args, _Problem(8, (5, 5, 1), 75))["rsvd_cols"] == 112
    assert bench.eig_kwargs(args, _Problem(4, (5, 5, 1), 5))["rsvd_cols"] == 13
    assert bench.eig_kwargs(args, _Problem(2, (3, 3, 1), 15))["rsvd_cols"] == 18   # capped at n = 18


def test_traffic_table_names_real_workloads_and_classes():
    workloads = {v[0] for v in bench.WORKLOADS.values()}
    classes = set(bench.KERNEL_NAMES.values())
    for (wl, cls), nbytes in bench.NCU_TRAFFIC.items():
        assert wl in workloads, wl
        assert cls in classes, cls
        assert isinstance(nbytes, int) and nbytes > 0


class _Stage:
    def __init__(self, ext, iters, gd_steps=1, p=1, off=(0, 0, 0)):
        self.off, self.ext, self.iters, self.gd_steps, self.p = off, ext, iters, gd_steps, p


class _Recon:
    def __init__(self, ncoil, kernel, circular, rank, stages):
        self.ncoil, self.kernel, self.circular, self.rank, self.stages = ncoil, kernel, circular, rank, stages


def test_gram_flops_follow_the_previous_iterations_region():
    # the Gram of outer iteration i is taken on the region of iteration i - 1 (the first stage's
    # region for the first iteration): a stage's first Gram is on the previous stage's region
    per_point = 8.0 * 2 * 2 * 5 ** 3 / 2          # C = 2, kernel 3 x 3 x 3: (2k-1)^3 lags
    centre, full = 8 * 8 * 4, 16 * 16 * 8
    pb = _Recon(2, (3, 3, 3), (0, 0, 0), 5,
                [_Stage((8, 8, 4), 2), _Stage((12, 12, 6), 0), _Stage((16, 16, 8), 3)])
    # iterations: centre, centre | (none) | centre (the last iteration's region), full, full
    assert bench.algorithmic_flops(pb, 0) == per_point * (3 * centre + 2 * full)


def test_step_flops_count_valid_outputs():
    # two convolutions and one adjoint per descent step, 8 n p s flops each; s counts the valid
    # outputs (ext - k + 1 per axis, the whole extent on a circular axis)
    pb = _Recon(2, (3, 3, 3), (0, 0, 1), 5, [_Stage((10, 9, 6), 2, gd_steps=3, p=4)])
    n, s = 2 * 27, 8 * 7 * 6
    assert bench.algorithmic_flops(pb, 6) == 2 * 3 * 2 * 8.0 * n * 4 * s
    assert bench.algorithmic_flops(pb, 7) == 2 * 3 * 8.0 * n * 4 * s
    assert bench.algorithmic_flops(pb, 8) == 2 * 16.0 * n ** 3 / 3.0


def test_class_roofline_against_the_pipe_of_the_class():
    pb = _Recon(2, (3, 3, 3), (0, 0, 0), 5, [_Stage((10, 9, 6), 2, gd_steps=3, p=4)])
    peaks = {"bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2000.0}
    conv = bench.class_roofline(pb, "none", 6, 2.0, 12, 1, peaks)
    assert conv["bound"] == "tensor" and conv["traffic"] is None
    assert abs(conv["achieved"] - bench.algorithmic_flops(pb, 6) / 2e-3 / 1e12) < 1e-12
    assert abs(conv["frac"] - conv["achieved"] / 1700.0) < 1e-15
    gram = bench.class_roofline(pb, "none", 0, 1.0, 2, 1, peaks)
    # double-word FP32 rate: 152 SMs x 128 lanes x clock / 40 operations per complex MAC x 8 flops
    assert abs(gram["peak"] - 152 * 128 * 2000e6 / 40 * 8 / 1e12) < 1e-9
    tri = bench.class_roofline(pb, "none", 8, 3.0, 2, 1, peaks)
    assert tri["bound"] == "latency" and tri["frac"] is None
    assert abs(tri["achieved"] - 1.5e3 / (54 - 2)) < 1e-9   # us per Householder step, n = 54
