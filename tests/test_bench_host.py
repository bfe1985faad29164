"""Host logic of the benchmark that the roofline figures rest on, on CPU:
the algorithmic bytes per launch of each kernel slot on the 1024x512 sheet
(64 particles per cell and species, FP32), the source hash that decides
whether a committed DRAM-traffic record still applies, and the oracle
sample that the CPU baseline times."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


NX, NY, PPC = 1024, 512, 64
NCELL = NX * NY
NSP = NCELL * PPC            # particles of one species
NPART = 2 * NSP


def test_algorithmic_bytes_of_the_headline_workload():
    # the push and the re-sort move one species' 24-byte records in and out
    # plus the run tables (18 and 19 int32 per cell); the deposit reads both
    # species' records and writes M (45 values) and Jhat (3) per node
    assert bench.algorithmic_bytes("push", NPART, NSP, NCELL, 4) == NSP * 48 + NCELL * 72 == 1648361472
    assert bench.algorithmic_bytes("permute", NPART, NSP, NCELL, 4) == NSP * 48 + NCELL * 76
    assert bench.algorithmic_bytes("deposit", NPART, NSP, NCELL, 4) == NPART * 24 + NCELL * 48 * 4
    # the operator: M in the form's precision, FP64-slot input and output
    assert bench.algorithmic_bytes("gmres_apply", NPART, NSP, NCELL, 4) == NCELL * (180 + 48)
    assert bench.algorithmic_bytes("unknown", NPART, NSP, NCELL, 4) is None


def test_source_hash_covers_device_code_only(tmp_path):
    dev = "namespace relsim {\nnamespace {\n__global__ void k() {}\n}  // namespace\n"
    host = "int launch() { return 0; }\n}\n"
    a = tmp_path / "a.cu"
    a.write_text(dev + host)
    h0 = bench.kernel_source_hash(str(a))
    a.write_text(dev + host.replace("0", "1"))
    assert bench.kernel_source_hash(str(a)) == h0          # a host-side edit keeps the record
    a.write_text(dev.replace("k()", "k2()") + host)
    assert bench.kernel_source_hash(str(a)) != h0          # a kernel edit voids it
    assert len(h0) == 16


def test_traffic_records_name_existing_sources():
    import json
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    for key, rec in d.items():
        if key.startswith("_"):
            continue
        src = os.path.join(ROOT, "paper_2509_11100_gb300", "csrc", rec["source"])
        assert os.path.exists(src), key
        assert rec["dram_bytes_per_launch"] > 0
        # the record is the capture scaled by the units of a full launch (x4)
        mb = rec["captured_read_mb"] + rec["captured_write_mb"]
        assert abs(rec["dram_bytes_per_launch"] - 4e6 * mb) <= 4e6 * 1e-3, key


def test_oracle_sample_keeps_every_kth_particle_of_each_cell_with_scaled_weights():
    from relsim_inputs import HarrisConfig, make_harris
    st = make_harris(HarrisConfig(nx=16, ny=8, ppc=16, seed=3))
    sub = bench.subsample(st, 8)
    for s0, s1 in zip(st["species"], sub["species"]):
        assert len(s1["w"]) * 8 == len(s0["w"])
        np.testing.assert_allclose(np.sum(s1["w"]), np.sum(s0["w"]), rtol=0.3)
        np.testing.assert_allclose(np.asarray(s1["w"]), 8 * np.asarray(s0["w"])[::8], rtol=0, atol=0)
