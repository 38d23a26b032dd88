"""Host-side pieces of bench.py that need no GPU: the fixed-tuning option and the
algorithmic byte counts the roofline divides by."""
import pytest

import bench


def test_parse_tuning_reads_names_and_numbers():
    assert bench.parse_tuning("tma_tiles=1, col_chunk=32,omega=0.65") == {"tma_tiles": 1, "col_chunk": 32,
                                                                        "omega": 0.65}
    assert bench.parse_tuning("") == {}
    with pytest.raises(SystemExit):
        bench.parse_tuning("tma_tiles")


def test_parse_tuning_names_are_set_tuning_keywords():
    import inspect
    from paper_1909_03948_gb300.hp import Problem, Tuning
    keywords = set(inspect.signature(Problem.set_tuning).parameters) - {"self"}
    assert keywords == {f for f, _ in Tuning._fields_}


def test_family_bytes_medium2d_smoothing_sweep():
    # 257^2 nodes, 60 FP32 columns: x and b read, y written (3 x 60 x 4 bytes per node)
    # plus diag, inverse diag and the two forward couplings (4 x 4 bytes per node)
    n = 257 * 257
    assert bench.family_bytes("smooth", n, 60, 2, True) == n * (720 + 16) == 48_612_064
    # 65^3 nodes, three forward couplings in 3D
    assert bench.family_bytes("smooth", 65 ** 3, 120, 3, True) == 65 ** 3 * (1440 + 20)


def test_level0_kernel_kind_follows_the_tile_shapes():
    on = {"tma_tiles": 1}
    assert bench.level0_kernel_kind(2, 256, on, True) == "tiled"
    assert bench.level0_kernel_kind(2, 256, {"tma_tiles": 0}, True) == "row"
    assert bench.level0_kernel_kind(2, 256, on, False) == "row"      # the tiled kernels are FP32
    assert bench.level0_kernel_kind(2, 16, on, True) == "row"        # narrower than one tile
    assert bench.level0_kernel_kind(3, 64, on, True) == "tiled"
    assert bench.level0_kernel_kind(3, 40, on, True) == "row"        # 40 is no multiple of the 32-wide tile


def test_traffic_records_belong_to_the_kernel_form_that_ran(tmp_path):
    # a record taken on one kernel form is never reported for the other, nor once that
    # form's source has changed since the capture
    import json
    rec = {"medium2d": {"smooth": {"dram_bytes_per_launch": 111, "kind": "row",
                                   "src_sha256": bench.stencil_kernel_sha256("row")}},
           "cube3d": {"smooth": {"dram_bytes_per_launch": 222, "kind": "tiled",
                                 "src_sha256": bench.stencil_kernel_sha256("tiled")},
                      "resid_mg": {"dram_bytes_per_launch": 333, "kind": "tiled", "src_sha256": "0" * 64}}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    assert bench.traffic_record("smooth", "medium2d", "row", str(p)) == 111
    assert bench.traffic_record("smooth", "medium2d", "tiled", str(p)) is None
    assert bench.traffic_record("smooth", "cube3d", "tiled", str(p)) == 222
    assert bench.traffic_record("smooth", "cube3d", "row", str(p)) is None
    assert bench.traffic_record("resid_mg", "cube3d", "tiled", str(p)) is None
    assert bench.traffic_record("matvec", "cube3d", "tiled", str(p)) is None


def test_the_two_kernel_forms_hash_different_sources():
    assert bench.stencil_kernel_sha256("row") != bench.stencil_kernel_sha256("tiled")


def test_cpu_baseline_states_its_sample_and_cores():
    import workloads as W
    cpu = bench.cpu_baseline_block(W.WORKLOADS["small2d"])
    assert cpu["value"] > 0 and cpu["kind"] == "oracle"
    assert cpu["cores"] == 1 and cpu["host_cores"] >= 1
    assert "1 thread of" in cpu["sample"] and "extrapolated" in cpu["sample"]


def test_3d_workload_oracle_solves_iteratively():
    # at 64^3 a sparse direct factorisation does not finish in minutes: the oracle's solves
    # (and so both CPU legs of the benchmark) are Jacobi-preconditioned CG there
    import workloads as W
    from oracle.inverse import CG_NODES_3D
    assert W.WORKLOADS["cube3d"].nnodes > CG_NODES_3D
    assert W.WORKLOADS["medium2d"].dim == 2


def test_committed_sweep_traffic_belongs_to_the_committed_kernel():
    # the cube3d z-march sweep's DRAM traffic in profiles/traffic.json was captured on the
    # kernel source as it stands: a kernel change without a new capture fails here
    assert bench.traffic_record("smooth", "cube3d", "tiled") is not None


def test_build_record_names_the_machine_and_compiler():
    rec = bench.build_record()
    assert rec["machine"]
    assert ("built_on" in rec and "nvcc" in rec and "lib_mtime" in rec) or "error" in rec
