"""Host-side logic of the autotuner: cache round trip and candidate lists."""
from paper_1609_04493_gb300 import autotune, binding as b


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("RDYN_TUNE_CACHE", str(tmp_path / "sub" / "tune.json"))
    autotune._store("k1", {"variant": 3})
    autotune._store("k2", {"variant": 5})
    c = autotune._load_cache()
    assert c["k1"]["variant"] == 3 and c["k2"]["variant"] == 5


def test_rnea_candidates_respect_lane_capacity():
    for n in (1, 16, 40, 100, 128):
        for v in autotune.rnea_candidates(n, 1024, None):
            if (v & 0xf00) == 0x100:
                assert n <= 8 * (v & 0xff)


def test_fleet_candidates_fit_a_cta():
    """Bits 0..7 of the tune word: blocks per SM; 8..15: log2 threads per block;
    16..23: the chain length from which forward-dynamics groups take two warps
    (such blocks hold whole warp pairs, at most 7 of them); bit 24: three warps
    instead (2^t / 64 triples per block, one or two)."""
    pairs = triples = 0
    for sched, tune in autotune.fleet_candidates():
        if sched == b.RD_SCHED_PERSISTENT:
            threads = 1 << ((tune >> 8) & 0xff)
            assert threads * (tune & 0xff) <= 1024
            length = (tune >> 16) & 0xff
            if tune >> 24:
                triples += 1
                assert threads in (64, 128) and length > 0
                assert tune == b.RD_FLEET_TUNE((tune >> 8) & 0xff, tune & 0xff) | \
                    b.RD_FLEET_THREE_WARPS(length)
            elif length:
                pairs += 1
                assert threads % 64 == 0 and threads <= 448
                assert tune == b.RD_FLEET_TUNE((tune >> 8) & 0xff, tune & 0xff) | \
                    b.RD_FLEET_TWO_WARPS(length)
    assert pairs and triples


def test_rnea_candidates_hybrid_store_fewer_links_than_the_chain():
    """Partial-state candidates keep state for fewer links than the chain has
    (K >= n is the stored kernel, already a candidate) and encode K / 4 in
    bits 20..27."""
    for n in (6, 16, 32, 100):
        hy = [v for v in autotune.rnea_candidates(n, 65536, None)
              if (v & 0xfff) == b.RD_VARIANT_SERIAL_HYBRID]
        assert hy, n
        for v in hy:
            K = 4 * ((v >> 20) & 0xff)
            assert 0 < K < n
            assert ((v >> 16) & 0xf) in (5, 6)  # 32 or 64 threads


def test_rnea_candidates_cover_the_common_normal_kernels():
    """Stored-prefix lengths never exceed the chain; the tensor-memory variant is
    offered only where it runs (FP32, n <= 32, n % 4 == 0)."""
    for n, dt in ((8, "float32"), (32, "float32"), (32, "float64"), (36, "float32"), (100, None)):
        cands = autotune.rnea_candidates(n, 65536, dt)
        dh = [v for v in cands if (v & 0xfff) == b.RD_VARIANT_SERIAL_DH]
        assert dh and all(4 * ((v >> 20) & 0xff) <= n for v in dh)
        tm = [v for v in cands if (v & 0xfff) == b.RD_VARIANT_SERIAL_DH_TMEM]
        assert bool(tm) == (n <= 32 and n % 4 == 0 and dt != "float64"), (n, dt)
        assert b.RD_VARIANT_AUTO in cands
