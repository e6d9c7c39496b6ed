"""Host logic of bench.py that needs no GPU: the pass-kernel code hash that keys the ncu
traffic table ignores comments and blank lines but not code, and the traffic lookup answers
only for the captured workload and precision."""
import os
import shutil

import bench


def _copy_sources(root):
    import pathlib
    src = os.path.join(bench.ROOT, "paper_2604_09233_gb300", "csrc")
    dst = pathlib.Path(root) / "paper_2604_09233_gb300" / "csrc"
    dst.mkdir(parents=True)
    for name in ("sense_tcp.cu", "sense_ptx.cuh", "sense_tc.cuh"):
        shutil.copy(os.path.join(src, name), dst / name)
    return dst


def test_pass_kernel_hash_ignores_comments_but_not_code(repo_tmp, monkeypatch):
    dst = _copy_sources(repo_tmp)
    monkeypatch.setattr(bench, "ROOT", str(repo_tmp))
    h0 = bench.pass_kernel_source_hash()
    f = dst / "sense_tcp.cu"
    text = f.read_text()
    anchor = "__global__ void __launch_bounds__(NTHREADS, 1) tcp_pass_kernel(Params p) {"
    assert anchor in text
    f.write_text(text.replace(anchor, "// an added comment\n\n" + anchor + "  // trailing"))
    assert bench.pass_kernel_source_hash() == h0
    f.write_text(text.replace("const uint16_t M1 = 0xBC00u;", "const uint16_t M1 = 0xBC01u;", 1))
    assert bench.pass_kernel_source_hash() != h0
    # the shared PTX wrappers are part of the kernel too
    f.write_text(text)
    w = dst / "sense_ptx.cuh"
    wt = w.read_text()
    w.write_text(wt.replace("(1024 >> 4) << 32", "(2048 >> 4) << 32", 1))
    assert bench.pass_kernel_source_hash() != h0


def test_traffic_lookup_is_specific_to_the_captured_case():
    recs = bench.KERNEL_TRAFFIC.get(bench.pass_kernel_source_hash())
    if recs is None:
        # the kernel changed since the last capture: every lookup reports no traffic
        assert bench._kernel_traffic("2d_256x256_32coil_35750samp_sh3", "tc_split",
                                     "tc_adjoint_pass") is None
        return
    for wl, rec in recs.items():
        prec = rec["precision"]
        assert bench._kernel_traffic(wl, prec, "tc_adjoint_pass") == rec["tc_adjoint_pass"]
        assert bench._kernel_traffic(wl, "tc_fp16", "tc_adjoint_pass") is None
    assert bench._kernel_traffic("another_workload", "tc_split", "tc_adjoint_pass") is None


def test_golden_cg_reader_matches_the_stored_text():
    """The bench's reader of the stored FP64 CG iterates returns every stored voxel and
    iteration count, with values equal to the text and norms equal to the header's norms
    scaled by the sampled fraction (every 64th voxel of a smooth image: same order of size)."""
    import numpy as np
    g = bench.golden_cg("2d_256x256_32coil_35750samp_sh3")
    assert g is not None
    assert list(g["voxels"][:3]) == [0, 64, 128] and len(g["voxels"]) == 65536 // 64
    assert sorted(g["iterates"]) == [5, 10, 40]
    path = bench.GOLDEN_CG["2d_256x256_32coil_35750samp_sh3"]
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert g["iterates"][40][7] == complex(float(rows[7][5]), float(rows[7][6]))
    head = [ln for ln in open(path) if ln.startswith("# norms")][0]
    full = {int(t.split(":")[0]): float(t.split(":")[1]) for t in head.split(":", 1)[1].split()}
    for n, v in g["iterates"].items():
        sampled = np.linalg.norm(v) * np.sqrt(64.0)
        assert 0.5 < sampled / full[n] < 2.0
    assert bench.golden_cg("another_workload") is None
