"""Host logic of the benchmark, on CPU: the algorithmic bytes per node behind every roofline
fraction it reports, the rule that a stored DRAM capture is reported only while the kernel sources
hash to the captured ones, and the bounded CPU-baseline sample of the oracle."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_per_node():
    b = _bench()
    # populations read and written (Q*K values), u* as 8 bytes per component read and written, flags
    assert b.bytes_per_node(3, 4) == 2 * 72 * 4 + 2 * 3 * 8 + 1 == 625
    assert b.bytes_per_node(3, 2) == 337          # BF16 storage
    assert b.bytes_per_node(3, 8) == 1201         # FP64 form
    assert b.bytes_per_node(2, 4) == 2 * 24 * 4 + 2 * 2 * 8 + 1
    # reverse step: gbar read and written, F and dL/du* read, dL/dmu (FP64) read and written, flags
    assert b.adjoint_bytes_per_node(3, 4) == 576 + 36 + 12 + 16 + 1 == 641
    assert b.recompute_bytes_per_node(3, 4) == 625 + 36
    # Jacobi sweep: correction vector (padded to 4) read and written, residual vector (FP64: flags)
    assert b.jacobi_bytes_per_node(3, 4) == 2 * 4 * 4 + 4 * 4 == 48
    assert b.jacobi_bytes_per_node(3, 4, 2) == 24
    assert b.jacobi_bytes_per_node(2, 4, 2) == (2 * 2 * 4 + 4 * 4) / 2
    assert b.jacobi_bytes_per_node(2, 4) == 2 * 2 * 4 + 4 * 4 + 1 == 33
    assert b.jacobi_bytes_per_node(3, 8) == 2 * 4 * 8 + 4 * 8 + 1
    # the method's figure: u* in the population precision (the coverage contract's 601 B in 3D FP32)
    assert b.method_bytes_per_node(3, 4) == 601
    assert b.method_bytes_per_node(3, 2) == 2 * 72 * 2 + 2 * 3 * 2 + 1
    assert b.method_bytes_per_node(2, 4) == 209
    # link kernel: per link 16 B of indices, 8 (1 + 3D) B of FP64 geometry, 3K + 2D values; per
    # stencil entry an index and D - 1 weights
    assert b.link_bytes(3, 4, 1, 0) == 16 + 8 * 10 + (36 + 6) * 4
    assert b.link_bytes(3, 4, 0, 10) == 10 * (4 + 8)


def test_traffic_is_reported_only_for_the_captured_sources():
    b = _bench()
    cur = b.kernel_sources_hash(b.KERNEL_SOURCES)
    cap = {"sources_sha256": cur, "bytes_per_launch": 1000, "windows": 40}
    # scaled by windows from the captured launch to the timed one
    assert b.captured_traffic(40, cap, b.KERNEL_SOURCES) == 1000
    assert b.captured_traffic(100, cap, b.KERNEL_SOURCES) == 2500
    # a capture of the timed size itself is reported as it is
    assert b.captured_traffic(None, dict(cap, windows=None), b.KERNEL_SOURCES) == 1000
    stale = dict(cap, sources_sha256="0" * 64)
    assert b.captured_traffic(40, stale, b.KERNEL_SOURCES) is None            # other sources
    assert b.captured_traffic(40, None, b.KERNEL_SOURCES) is None
    # the stored captures are either current or reported as null
    for c, src in ((b.TRAFFIC_CAPTURE, b.KERNEL_SOURCES), (b.BF16_TRAFFIC_CAPTURE, b.KERNEL_SOURCES),
                   (b.ADJ_TRAFFIC_CAPTURE, b.ADJ_SOURCES)):
        if c:
            got = b.captured_traffic(c.get("windows") or None, c, src)
            assert got in (None, c["bytes_per_launch"])
    # the hash covers every listed source: dropping one changes it
    assert b.kernel_sources_hash(b.KERNEL_SOURCES[:-1]) != b.kernel_sources_hash(b.KERNEL_SOURCES)


def test_oracle_sample_is_bounded_and_whole_projection_cycles():
    b = _bench()
    for threads in (1, 0):
        mlups, steps, elapsed, nact = b.oracle_sample(n=16, budget_s=0.5, threads=threads)
        assert steps >= 20 and steps % 20 == 0
        assert nact > 0 and mlups > 0 and elapsed < 30
