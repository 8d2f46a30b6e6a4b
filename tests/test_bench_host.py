"""Host logic of the benchmark (no GPU): the keyword parameters and initial fields of every
workload, and the rule that an ncu traffic figure is reported only while the sources it was
captured on are unchanged."""
import numpy as np
import pytest

import bench
from paper_2106_07694_gb300 import lbm_wenoc as lw, workloads


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_workload_parameters_are_accepted_by_the_boundary(name):
    wl = bench.WORKLOADS[name][0]
    p = lw.make_params(wl.shape, fp64=wl.dtype == "f64", **bench.phys_kwargs(wl))
    assert lw.lbm_wenoc_workspace_bytes(p) > 0


def test_variant_and_class_workloads():
    assert bench.phys_kwargs(workloads.WENO3_2D)["weno3"] is True
    assert bench.phys_kwargs(workloads.SIGN_SPLIT_2D)["sign_split"] is True
    kw = bench.phys_kwargs(workloads.CLASSES_2D)
    assert kw["class_vs"] == workloads.CLASSES_2D.class_vs and len(kw["class_vs"]) == 3
    assert "class_vs" not in bench.phys_kwargs(workloads.MAIN_2D)
    # the classes share the interface field: their sum is the single-class field
    small = workloads.CLASSES_2D.with_(shape=(64, 32))
    total = sum(small.initial_classes())
    assert np.allclose(total, small.initial_c(), rtol=1e-15, atol=1e-15)

    class Recorder:
        def __init__(self):
            self.calls = []

        def set_class(self, k, ck):
            self.calls.append((k, ck.shape))

    r = Recorder()
    bench.set_classes(r, small)
    assert [k for k, _ in r.calls] == [0, 1, 2]
    r2 = Recorder()
    bench.set_classes(r2, workloads.MAIN_2D)
    assert r2.calls == []


def test_traffic_is_reported_only_for_unchanged_sources(monkeypatch):
    name = "lbm_collide_stream"
    nbytes, files, _ = bench.NCU_TRAFFIC[name]
    sha = bench.source_hash(files)
    monkeypatch.setitem(bench.NCU_TRAFFIC, name, (nbytes, files, sha))
    assert bench.kernel_traffic(name) == nbytes  # a capture taken on the current sources
    monkeypatch.setitem(bench.NCU_TRAFFIC, name, (nbytes, files, "0" * 12))
    assert bench.kernel_traffic(name) is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, name, (nbytes, ("no_such_file.cuh",), sha))
    assert bench.kernel_traffic(name) is None
    assert bench.kernel_traffic("not_a_kernel") is None


def test_traffic_of_the_3d_workload_comes_from_its_own_table(monkeypatch):
    name = "rk_stage1"
    nb2, files2, _ = bench.NCU_TRAFFIC[name]
    nb3, files3, _ = bench.NCU_TRAFFIC_3D[name]
    assert nb3 != nb2 and files3[0].startswith("transport_sweep3d")
    monkeypatch.setitem(bench.NCU_TRAFFIC_3D, name, (nb3, files3, bench.source_hash(files3)))
    assert bench.kernel_traffic(name, bench.NCU_TRAFFIC_3D) == nb3
    monkeypatch.setitem(bench.NCU_TRAFFIC_3D, name, (nb3, files3, "f" * 12))
    assert bench.kernel_traffic(name, bench.NCU_TRAFFIC_3D) is None
