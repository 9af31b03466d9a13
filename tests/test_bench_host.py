"""Host logic of bench.py: the kernel-code fingerprint that keys a committed
DRAM-traffic capture, and the lookup of that capture."""
import os
import shutil

import bench


def copy_tree(tmp_path):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1612_08312_gb300", "csrc"),
                    root / "paper_1612_08312_gb300" / "csrc",
                    ignore=shutil.ignore_patterns("*.o", "*.so"))
    (root / "profiles").mkdir()
    return root


def fingerprint(root):
    old = bench.ROOT
    bench.ROOT = str(root)
    try:
        return bench.kernel_source_hash()
    finally:
        bench.ROOT = old


def test_fingerprint_ignores_comments_and_whitespace_but_not_code(tmp_path):
    root = copy_tree(tmp_path)
    base = fingerprint(root)
    f = root / "paper_1612_08312_gb300" / "csrc" / "ising.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n/* and a block\n   comment */\n" + text.replace("\n", "\n\n", 3))
    assert fingerprint(root) == base
    f.write_text(text.replace("MEASURE_BLOCK = 128", "MEASURE_BLOCK = 64"))
    assert fingerprint(root) != base
    f.write_text(text)
    g = root / "paper_1612_08312_gb300" / "csrc" / "graph.cu"
    g.write_text(g.read_text().replace("GB_THREADS = 256", "GB_THREADS = 128"))
    assert fingerprint(root) == base  # another model's kernels


def test_committed_traffic_is_read_per_kernel_and_fingerprint(tmp_path):
    root = copy_tree(tmp_path)
    h = fingerprint(root)
    (root / "profiles" / "traffic.txt").write_text(
        "# kernel bytes_per_site source_hash\n"
        f"ising_local_kernel 2.5 {h}\n"
        "ising_flip_kernel 3.0 0000000000000000\n")
    old = bench.ROOT
    bench.ROOT = str(root)
    try:
        assert bench.committed_traffic("ising_local_kernel", 1000) == 2500.0
        assert bench.committed_traffic("ising_flip_kernel", 1000) is None  # taken on other code
        assert bench.committed_traffic("ising_measure_kernel", 1000) is None
    finally:
        bench.ROOT = old


def test_generic_workload_inputs_and_bytes():
    """The generic-lattice workloads' inputs: the explicit simple-cubic bond
    list handed to the library is the oracle's, site masks are seeded and
    have the stated occupation, and the algorithmic bytes per site follow
    the stated model (14 B, plus 8 B per listed bond)."""
    import numpy as np
    import oracle
    import workloads
    for L in (3, 4, 6):
        a = workloads.sc_bond_list(L)
        b = oracle.sc_edges(L)
        assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    m1 = workloads.site_mask(100000, 0.8, 7)
    m2 = workloads.site_mask(100000, 0.8, 7)
    assert (m1 == m2).all() and abs(m1.mean() - 0.8) < 0.01 and m1.dtype == np.uint8
    assert bench.graph_bytes_per_site(bench.WORKLOADS["sc_L640"]) == 14.0
    assert bench.graph_bytes_per_site(bench.WORKLOADS["sc_list_L512"]) == 14.0 + 24.0
    for name in ("sc_L640", "sc_dil_L512", "sc_list_L512"):
        wl = bench.WORKLOADS[name]
        assert wl["model"] == 1 and wl["lattice"] in ("sc", "list")
    # the simple-cubic L = 640 lattice has about the pyrochlore L = 256 site count
    assert abs(640 ** 3 / (16 * 256 ** 3) - 1) < 0.03
