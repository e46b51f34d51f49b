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
