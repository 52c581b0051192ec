"""GPU parity: the CUDA path against the CPU oracle, element by element, on the
same seeded inputs.  Integer work throughout, so everything must be bit-exact:
master hashes, partition order, pilots, every packed word of the structure,
bits/key and every query output."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18497_b300 import build, phobic

    build.build()
    phobic.lib()
    return phobic


def _dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def _keys(n, seed):
    from paper_2404_18497_b300 import workloads

    return workloads.distinct_u64(n, seed)


def compare_structure(ph, orc_h, h, encoder):
    """Every array of the exported structure equals the oracle's.  A mono encoder
    (5..8) has its column encoder's arrays for a single column."""
    ex = ph.parse_export(ph.phobic_export(h))
    assert ex["encoder"] == encoder
    encoder = encoder - 5 if encoder >= 5 else encoder
    o = orc_h
    assert ex["n"] == o.u64("n") and ex["M"] == o.u64("M") and ex["NP"] == o.u64("NP") and ex["B"] == o.u64("B")
    assert ex["off_w"] == o.u64("off_w") and ex["off_Q"] == o.u64("off_Q") and ex["off_dmin"] == o.u64("off_dmin")
    assert (ex["off_words"] == o.array("off_words")).all()
    meta = ex["col_meta"]
    mask = np.uint64((1 << 56) - 1)
    if encoder == 0:
        assert ((meta >> np.uint64(56)).astype(np.uint32) == o.array("col_w")).all()
        assert ((meta & mask) == o.array("col_base")).all()
        assert (ex["pil_words"] == o.array("pil_words")).all()
    elif encoder in (2, 3, 4):
        assert ((meta[0::2] >> np.uint64(56)).astype(np.uint32) == o.array("col_l")).all()
        assert ((meta[0::2] & mask) == o.array("col_lbase")).all()
        assert (meta[1::2] == o.array("col_hbase")).all()
        assert (ex["pil_words"] == o.array("rice_low")).all()
        assert (ex["rice_high"] == o.array("rice_high")).all()
        assert (ex["rice_samples"] == o.array("rice_samples")).all()
    else:
        assert ((meta[0::2] >> np.uint64(56)).astype(np.uint32) == o.array("col_rw")).all()
        assert ((meta[0::2] & mask) == o.array("col_rbase")).all()
        assert ((meta[1::2] >> np.uint64(56)).astype(np.uint32) == o.array("col_dw")).all()
        assert ((meta[1::2] & mask) == o.array("col_dbase")).all()
        assert (ex["pil_words"] == o.array("rank_words")).all()
        assert (ex["dict_words"] == o.array("dict_words")).all()
    if o.u64("ef_N"):
        assert ex["ef_l"] == o.u64("ef_l")
        assert (ex["ef_low"] == o.array("ef_low")).all()
        assert (ex["ef_high"] == o.array("ef_high")).all()
        assert (ex["ef_samples"] == o.array("ef_samples")).all()
    else:
        assert ex["n_ef_low"] == 0 and ex["n_ef_high"] == 0
    for k in ["bits_header", "bits_offsets", "bits_pilots", "bits_remap", "bits_total"]:
        assert ex[k] == o.u64(k), k


def test_master_hash_parity(ph, orc):
    keys = _keys(1_000_003, 1)
    for seed in (0, 1, 0xDEADBEEF):
        got = _host(ph.phobic_hash_u64(_dev(keys), seed))
        assert (got == orc.key_hash(keys, seed)).all()
    # 8- but not 16-byte aligned input and output (the kernel's scalar path), odd and tiny lengths
    buf = torch.zeros(keys.size + 1, dtype=torch.int64, device="cuda")
    buf[1:] = _dev(keys)
    out = torch.zeros(keys.size + 1, dtype=torch.int64, device="cuda")
    ph.phobic_hash_u64(buf[1:], 5, out[1:])
    assert (_host(out[1:]) == orc.key_hash(keys, 5)).all()
    for m in (1, 2, 3):
        assert (_host(ph.phobic_hash_u64(_dev(keys[:m]), 5)) == orc.key_hash(keys[:m], 5)).all()


def test_string_hash_parity(ph, orc):
    from paper_2404_18497_b300 import workloads

    data, off = workloads.random_strings(200_001, 5, 0, 70)
    got = _host(ph.phobic_hash_strings(torch.from_numpy(data).cuda(), _dev(off), 7))
    assert (got == orc.string_hashes(data, off, 7)).all()


def test_string_hash_known_answers(ph):
    """The device XXH64 against published known answers (the same fixture that
    pins the oracle), every path of the hash: tails of 1-7 bytes, 8-byte lanes,
    one and several 32-byte stripes, nonzero seeds."""
    from tests import xxh64_known

    for seed, (data, offs, want) in xxh64_known.by_seed().items():
        got = _host(ph.phobic_hash_strings(torch.from_numpy(data).cuda(), _dev(offs), seed))
        assert [int(v) for v in got] == want, seed


@pytest.mark.parametrize("n,P", [(1, 2500), (100, 2500), (2500, 2500), (1_000_000, 2500), (1_234_567, 1000),
                                 (300_000, 37), (5_000_000, 2500), (65_536, 1), (3_000_000, 24),
                                 (1_000_000, 1), (2_000_000, 3)])
def test_partition_sort_parity(ph, orc, n, P):
    """Section 4: keys grouped by partition j = floor(hk N_P / 2^64), partitions
    ascending.  j is monotone in hk, so sorting each partition's segment must give
    the globally sorted hashes."""
    keys = _keys(n, n)
    hk = orc.key_hash(keys, 3)
    NP = orc.lib().or_num_partitions(n, P)
    srt, start = ph.phobic_partition_sort(_dev(hk), NP)
    srt, start = _host(srt), start.cpu().numpy()
    sizes = orc.partition_sizes(hk, min(7.0, P), 1.0, P)  # lambda does not change partitions
    assert (start == np.concatenate([[0], np.cumsum(sizes)])).all()
    seg = np.repeat(np.arange(NP), sizes.astype(np.int64))
    assert np.array_equal(srt[np.lexsort((srt, seg))], np.sort(hk))


CASES = [
    # n, lam, alpha, P, encoder, mode
    (1, 7.0, 1.0, 2500, 0, 0),
    (2, 7.0, 0.99, 2500, 1, 0),
    (100, 3.0, 1.0, 8, 0, 0),
    (2500, 7.0, 1.0, 2500, 0, 0),
    (2501, 7.0, 0.99, 2500, 1, 0),
    (10_007, 5.0, 0.9, 300, 1, 0),
    (20_000, 3.0, 1.0, 3, 0, 0),  # partitions of about 3 keys, one bucket each
    (50_000, 6.0, 0.7, 2500, 0, 0),
    (100_000, 7.0, 1.0, 2500, 0, 1),
    (100_000, 7.0, 0.99, 2500, 1, 1),
    (200_000, 8.0, 1.0, 4096, 1, 0),
    (300_000, 7.0, 0.99, 1024, 0, 0),
    (1_000_000, 7.0, 1.0, 2500, 0, 0),   # the 1M-key configuration (IC-C, alpha = 1)
    (1_000_000, 7.0, 0.99, 2500, 1, 0),  # the 1e8-key configuration's parameters at 1M keys
    # IC-R (interleaved Golomb-Rice)
    (1, 7.0, 1.0, 2500, 2, 0),
    (100, 3.0, 1.0, 8, 2, 0),
    (2501, 7.0, 0.99, 2500, 2, 0),
    (70_001, 6.0, 0.9, 300, 2, 1),
    (300_000, 9.0, 0.99, 1024, 2, 0),
    (1_000_000, 8.0, 1.0, 2500, 2, 0),
    (1_000_000, 7.0, 0.99, 2500, 2, 0),
    # IC-EF (interleaved Elias-Fano over each column's prefix sums)
    (1, 7.0, 1.0, 2500, 3, 0),
    (2501, 7.0, 0.99, 2500, 3, 0),
    (70_001, 6.0, 0.9, 300, 3, 1),
    (1_000_000, 8.0, 1.0, 2500, 3, 0),
    # the large-lambda regime (search cost ~ e^lambda per key, Section 3)
    (400_000, 10.0, 1.0, 2500, 2, 0),
    (150_000, 12.0, 1.0, 2500, 2, 0),
    (150_000, 11.0, 0.99, 2500, 0, 1),
]


@pytest.mark.parametrize("n,lam,alpha,P,enc,mode", CASES)
def test_build_and_query_parity(ph, orc, n, lam, alpha, P, enc, mode):
    keys = _keys(n, 17 + n)
    seed = 11
    o = orc.Oracle(keys, lam=lam, alpha=alpha, P=P, encoder=enc, mode=mode, seed=seed, threads=0)
    prm = ph.make_params(lam, alpha, P, seed=seed, encoder=enc, mode=mode, keep_pilots=True)
    dk = _dev(keys)
    h = ph.phobic_build_ex(dk, prm)
    info = h.info()
    assert info["n"] == n and info["M"] == o.u64("M") and info["num_partitions"] == o.u64("NP")
    # pilots
    gp = h.pilots().cpu().numpy().view(np.uint32)
    assert np.array_equal(gp, o.pilots)
    # packed structure and space
    compare_structure(ph, o, h, enc)
    assert h.bits_per_key() == o.bits_per_key()
    # every query, positive and negative
    got = _host(h.query(dk))
    ref = o.query(keys)
    assert np.array_equal(got, ref)
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint64))
    neg = np.random.default_rng(n).integers(0, 2**64, size=min(n, 50_000), dtype=np.uint64)
    assert np.array_equal(_host(h.query(_dev(neg))), o.query(neg))
    h.free()


@pytest.mark.parametrize("fn", [1, 2, 3])
@pytest.mark.parametrize("alpha,enc", [(1.0, 0), (0.99, 2)])
def test_ablation_bucket_functions_parity(ph, orc, fn, alpha, enc):
    """Figure 3a's other bucket assignment functions (beta_*, PTHash's skewed
    split, uniform): the same bit-exact structure and queries as the oracle, and
    the function survives export and import."""
    keys = _keys(150_000, 70 + fn)
    o = orc.Oracle(keys, lam=5.0, alpha=alpha, P=2500, encoder=enc, bucket_fn=fn, threads=0)
    h = ph.phobic_build_ex(_dev(keys), ph.make_params(5.0, alpha, 2500, encoder=enc, keep_pilots=True,
                                                      bucket_function=fn))
    assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots)
    compare_structure(ph, o, h, enc)
    assert h.info()["bucket_function"] == fn
    assert np.array_equal(_host(h.query(_dev(keys))), o.query(keys))
    h2 = ph.phobic_import(ph.phobic_export(h))
    assert h2.info()["bucket_function"] == fn
    assert torch.equal(h2.query(_dev(keys)), h.query(_dev(keys)))


@pytest.mark.parametrize("c", [0, 6, 40, 358, 400])
def test_compact_rice_mixture_parity(ph, orc, c):
    """Section 4.1's mixture (the first c columns Compact, the rest Golomb-Rice):
    bit-exact structure and queries for c from 0 (IC-R) to past B (IC-C), with
    alpha < 1 and both pilot modes, through export and import."""
    keys = _keys(400_000, 90 + c)
    for mode, alpha in [(0, 0.99), (1, 1.0)]:
        o = orc.Oracle(keys, lam=7.0, alpha=alpha, P=2500, encoder=4, mode=mode, compact_columns=c, threads=0)
        h = ph.phobic_build_ex(_dev(keys), ph.make_params(7.0, alpha, 2500, encoder=4, mode=mode,
                                                          compact_columns=c, keep_pilots=True))
        assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots)
        compare_structure(ph, o, h, 4)
        assert h.bits_per_key() == o.bits_per_key()
        assert h.info()["compact_columns"] == min(c, 358)
        assert np.array_equal(_host(h.query(_dev(keys))), o.query(keys))
        h2 = ph.phobic_import(ph.phobic_export(h))
        assert torch.equal(h2.query(_dev(keys)), h.query(_dev(keys)))
        h.free()


@pytest.mark.parametrize("enc", [5, 6, 7, 8])
def test_mono_encoder_parity(ph, orc, enc):
    """Section 5, Figure 3b: mono-C/D/R/EF place all pilots in one encoder.  The
    GPU keeps one work item per physical column and carries the set-wide width,
    dictionary, Rice parameter or Elias-Fano prefix across them; the structure is
    bit-exact with the oracle's one-column encoding, for alpha < 1 and both pilot
    modes, ragged partition counts, and through export and import."""
    keys = _keys(400_000 + 3 * enc, 110 + enc)
    for mode, alpha, P in [(0, 0.99, 2500), (1, 1.0, 1000), (0, 0.97, 4096)]:
        o = orc.Oracle(keys, lam=7.0, alpha=alpha, P=P, encoder=enc, mode=mode, threads=0)
        h = ph.phobic_build_ex(_dev(keys), ph.make_params(7.0, alpha, P, encoder=enc, mode=mode, keep_pilots=True))
        assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots)
        compare_structure(ph, o, h, enc)
        assert h.bits_per_key() == o.bits_per_key()
        assert np.array_equal(_host(h.query(_dev(keys))), o.query(keys))
        h2 = ph.phobic_import(ph.phobic_export(h))
        assert torch.equal(h2.query(_dev(keys)), h.query(_dev(keys)))
        h.free()


@pytest.mark.parametrize("enc", list(range(9)))
def test_import_of_oracle_written_files(ph, orc, enc):
    """A structure the library never built: the oracle's arrays written in the
    documented export layout.  Imported, the GPU query path answers every key
    (and non-members) exactly as the oracle does, and exports the same bytes."""
    import os
    import sys

    sys.path.insert(0, os.path.dirname(__file__))
    from oracle_export import oracle_export

    keys = _keys(300_000 + enc, 120 + enc)
    others = _keys(50_000, 999)
    for alpha, mode, P in [(0.99, 0, 2500), (1.0, 1, 1000), (0.95, 0, 4096)]:
        o = orc.Oracle(keys, lam=7.0, alpha=alpha, P=P, encoder=enc, mode=mode, compact_columns=9, seed=4, threads=0)
        data = oracle_export(o)
        h = ph.phobic_import(data)
        assert np.array_equal(_host(h.query(_dev(keys))), o.query(keys))
        assert np.array_equal(_host(h.query(_dev(others))), o.query(others))
        assert ph.phobic_export(h) == data
        h.free()


@pytest.mark.parametrize("enc", list(range(9)))
def test_tiny_sets_every_encoder(ph, orc, enc):
    """Degenerate sizes for every encoder (interleaved, mixture and mono): one
    key, a handful, exactly one partition and one key more; both pilot forms,
    with and without the Elias-Fano remap; bit-exact structure and queries."""
    for n in (1, 2, 3, 2500, 2501):
        keys = _keys(n, 500 + n + 10 * enc)
        for mode, alpha in ((0, 1.0), (1, 0.97)):
            o = orc.Oracle(keys, lam=7.0, alpha=alpha, P=2500, encoder=enc, mode=mode, compact_columns=3,
                           threads=0)
            h = ph.phobic_build_ex(_dev(keys), ph.make_params(7.0, alpha, 2500, encoder=enc, mode=mode,
                                                              compact_columns=3, keep_pilots=True))
            assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots), (n, mode)
            compare_structure(ph, o, h, enc)
            assert np.array_equal(_host(h.query(_dev(keys))), o.query(keys)), (n, mode)
            h.free()


def test_query_unaligned_and_odd_lengths(ph, orc):
    keys = _keys(30_001, 4)
    o = orc.Oracle(keys, lam=6.0, P=500, threads=0)
    h = ph.phobic_build(_dev(keys), 6.0, 1.0, 500, 0)
    buf = torch.zeros(30_002, dtype=torch.int64, device="cuda")
    buf[1:] = _dev(keys)
    out = torch.zeros(30_002, dtype=torch.int64, device="cuda")
    ph.phobic_query(h, buf[1:], out[1:])  # 8-byte but not 16-byte aligned
    assert np.array_equal(_host(out[1:]), o.query(keys))
    for m in (0, 1, 2, 3, 31):
        assert np.array_equal(_host(h.query(_dev(keys[:m]))) if m else np.zeros(0, np.uint64), o.query(keys[:m]))


def test_export_import_roundtrip(ph, orc):
    keys = _keys(123_457, 8)
    for enc, alpha in [(0, 1.0), (1, 0.95), (2, 0.99), (3, 0.99), (5, 1.0), (6, 0.99), (7, 0.99), (8, 1.0)]:
        h = ph.phobic_build_ex(_dev(keys), ph.make_params(7.0, alpha, 2500, encoder=enc))
        data = ph.phobic_export(h)
        h2 = ph.phobic_import(data)
        assert ph.phobic_export(h2) == data
        assert torch.equal(h.query(_dev(keys)), h2.query(_dev(keys)))
        assert h2.bits_per_key() == h.bits_per_key()
        bad = bytearray(data)
        bad[0] ^= 1
        with pytest.raises(ph.PhobicError) as e:
            ph.phobic_import(bytes(bad))
        assert e.value.status == "FORMAT"
        with pytest.raises(ph.PhobicError):
            ph.phobic_import(data[:-8])
        if enc in (2, 3, 7, 8):
            # a unary region with a missing one, or a wrong select sample, is refused
            ex = ph.parse_export(data)
            w = np.frombuffer(data, dtype=np.uint64).copy()
            hi0 = len(ph.HEADER_FIELDS) + sum(ex["n_" + a] for a in ph.ARRAYS[:3]) + (
                ex["n_dict_words"] - ex["rice_high"].size)
            nz = hi0 + int(np.flatnonzero(ex["rice_high"])[3])
            for flip_word, bit in [(nz, None), (hi0 - (ex["n_dict_words"] - ex["rice_high"].size), 40)]:
                bad = w.copy()
                if bit is None:
                    bad[flip_word] &= bad[flip_word] - np.uint64(1)  # clear the lowest set bit
                else:
                    bad[flip_word] ^= np.uint64(1) << np.uint64(bit)  # corrupt the second sample
                with pytest.raises(ph.PhobicError) as e:
                    ph.phobic_import(bad.tobytes())
                assert e.value.status == "FORMAT"


def test_errors(ph):
    keys = _keys(10_000, 9)
    dup = np.concatenate([keys, keys[5:6]])
    with pytest.raises(ph.PhobicError) as e:
        ph.phobic_build(_dev(dup), 7.0, 1.0, 2500, 0)
    assert e.value.status == "DUP_HASH"
    # every search variant reports the same errors (several warps per partition
    # keep the first final outcome in enumeration order)
    for mode in (0, 1):
        for wpp in (1, 2, 4, 8):
            with pytest.raises(ph.PhobicError) as e:
                ph.phobic_build_ex(_dev(dup), ph.make_params(7.0, 1.0, 2500, mode=mode, warps_per_partition=wpp))
            assert e.value.status == "DUP_HASH", (mode, wpp)
            with pytest.raises(ph.PhobicError) as e:
                ph.phobic_build_ex(_dev(keys), ph.make_params(12.0, 1.0, 2500, mode=mode, s_max=1,
                                                              warps_per_partition=wpp))
            assert e.value.status == "SEARCH_LIMIT", (mode, wpp)
    for wpp in (3, 16):
        with pytest.raises(ph.PhobicError) as e:
            ph.phobic_build_ex(_dev(keys), ph.make_params(7.0, 1.0, 2500, warps_per_partition=wpp))
        assert e.value.status == "INVALID_ARG"
    for kw in [dict(lam=0.0), dict(alpha=0.0), dict(alpha=1.5), dict(P=0), dict(P=100_000), dict(lam=9.0, P=8)]:
        args = dict(lam=7.0, alpha=1.0, P=2500)
        args.update(kw)
        with pytest.raises(ph.PhobicError) as e:
            ph.phobic_build_ex(_dev(keys), ph.make_params(**args))
        assert e.value.status == "INVALID_ARG"
    # a partition whose table reaches 2^16 slots (the search holds slots as u16):
    # P = 16384 at alpha = 0.2 gives m_j = ceil(n_j / 0.2) ~ 81920; the build
    # refuses it before any search launch (the oracle, with no such limit, builds it)
    big = _keys(4 * 16384, 12)
    for mode in (0, 1):
        with pytest.raises(ph.PhobicError) as e:
            ph.phobic_build_ex(_dev(big), ph.make_params(7.0, 0.2, 16384, mode=mode))
        assert e.value.status == "PARTITION_TOO_LARGE", mode
    # the context is still usable after the errors
    h = ph.phobic_build(_dev(keys), 7.0, 1.0, 2500, 0)
    assert torch.unique(h.query(_dev(keys))).numel() == keys.size


@pytest.mark.parametrize("mode", [0, 1])
def test_search_limit_matches_oracle(ph, orc, mode):
    """With a small s_max both sides fail (or succeed) on the same inputs, for
    every number of warps per partition."""
    keys = _keys(50_000, 10)
    for s_max in (1, 2, 4, 64):
        try:
            orc.Oracle(keys, lam=9.0, P=2500, mode=mode, s_max=s_max, threads=0)
            o_ok = True
        except orc.OracleError as e:
            assert e.code == orc.SEARCH_LIMIT
            o_ok = False
        for wpp in (1, 2, 4, 8):
            try:
                ph.phobic_build_ex(_dev(keys), ph.make_params(9.0, 1.0, 2500, mode=mode, s_max=s_max,
                                                              warps_per_partition=wpp)).free()
                g_ok = True
            except ph.PhobicError as e:
                assert e.status == "SEARCH_LIMIT"
                g_ok = False
            assert o_ok == g_ok, (s_max, wpp)


def test_host_entry_points(ph, orc):
    keys = _keys(77_777, 12)
    prm = ph.make_params(7.0, 0.99, 2500, encoder=1)
    h1 = ph.phobic_build_host(keys, prm)
    h2 = ph.phobic_build_ex(_dev(keys), prm)
    assert ph.phobic_export(h1) == ph.phobic_export(h2)
    out = ph.phobic_query_host(h1, keys)
    assert np.array_equal(out, _host(h2.query(_dev(keys))))
    # more than one 4M-key chunk: the pipelined path (slots reused, a ragged last chunk)
    big = np.random.default_rng(5).integers(0, 2**64, size=10_500_001, dtype=np.uint64)
    big[::3] = keys[np.arange(0, big.size, 3) % keys.size]
    out = ph.phobic_query_host(h1, big)
    assert np.array_equal(out, _host(h2.query(_dev(big))))


@pytest.mark.parametrize("mode,lam,P", [(0, 7.0, 2500), (1, 7.0, 2500), (0, 9.0, 1024), (1, 8.0, 4096)])
def test_search_variants_agree(ph, orc, mode, lam, P, monkeypatch):
    """Window width (32 or 64 displacements per lane), key placement (shared
    memory or global scratch), schedule (one CTA per partition or a work queue)
    and warps per partition change speed only: pilots equal the oracle's."""
    keys = _keys(200_000, 31)
    o = orc.Oracle(keys, lam=lam, alpha=0.99, P=P, mode=mode, threads=0)
    for in_smem in ("0", "1"):
        monkeypatch.setenv("PHOBIC_KEYS_IN_SMEM", in_smem)
        for width in (32, 64):
            for sched in (1, 2):
                for wpp in (1, 2, 4, 8):
                    h = ph.phobic_build_ex(_dev(keys), ph.make_params(lam, 0.99, P, mode=mode, keep_pilots=True,
                                                                      candidate_width=width, search_schedule=sched,
                                                                      warps_per_partition=wpp))
                    assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots), \
                        (in_smem, width, sched, wpp)
                    h.free()


@pytest.mark.parametrize("n,lam,alpha,enc", [(1, 7.5, 0.99, 0), (50_000, 7.5, 0.99, 1), (1_000_000, 7.5, 0.99, 1),
                                             (300_000, 7.0, 1.0, 0)])
def test_string_build_and_query_parity(ph, orc, n, lam, alpha, enc):
    """Section 5's input: random strings of length 10-50 over [A-Za-z0-9],
    reduced to XXH64 master hashes on the device; then the same construction."""
    from paper_2404_18497_b300 import workloads

    data, off = workloads.random_strings(n, 40 + n)
    hk = orc.string_hashes(data, off, 9)
    o = orc.Oracle(hashed=hk, lam=lam, alpha=alpha, P=2500, encoder=enc, seed=9, threads=0)
    dd, do = torch.from_numpy(data).cuda(), _dev(off)
    h = ph.phobic_build_strings(dd, do, ph.make_params(lam, alpha, 2500, seed=9, encoder=enc, keep_pilots=True))
    assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots)
    compare_structure(ph, o, h, enc)
    got = _host(ph.phobic_query_strings(h, dd, do))
    assert np.array_equal(got, o.query_hashed(hk))
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint64))
    # a string handle refuses 64-bit queries, and the other way round
    with pytest.raises(ph.PhobicError):
        ph.phobic_query(h, _dev(np.arange(4, dtype=np.uint64)))
    # export / import keeps the key kind
    h2 = ph.phobic_import(ph.phobic_export(h))
    assert np.array_equal(_host(ph.phobic_query_strings(h2, dd, do)), got)


def test_string_hash_unaligned_and_tails(ph, orc):
    """Strings at every byte alignment and every tail length, including the last
    bytes of the buffer (no read past offsets[n])."""
    rng = np.random.default_rng(77)
    lens = np.concatenate([np.arange(0, 80), rng.integers(0, 80, size=5000)])
    off = np.zeros(lens.size + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    data = rng.integers(0, 256, size=int(off[-1]), dtype=np.uint8)
    for shift in (0, 1, 3, 7):
        buf = torch.zeros(data.size + 8, dtype=torch.uint8, device="cuda")
        view = buf[shift:shift + data.size]
        view.copy_(torch.from_numpy(data))
        got = _host(ph.phobic_hash_strings(view, _dev(off), 123))
        assert np.array_equal(got, orc.string_hashes(data, off, 123))


@pytest.mark.parametrize("alpha,enc", [(0.99, 1), (1.0, 0), (0.99, 2), (1.0, 3), (1.0, 5), (0.99, 6), (0.99, 7),
                                       (1.0, 8)])
def test_batch_build_matches_single_builds(ph, orc, alpha, enc):
    """Batched construction: every set's structure equals the oracle's build of
    that set alone (and so the single-set path), for uneven set sizes and mixed
    partition sizes."""
    from paper_2404_18497_b300 import workloads

    rng = np.random.default_rng(123)
    sizes = np.concatenate([[1, 2, 3, 17, 2499, 2500, 2501], workloads.log_uniform_sizes(40, 10, 200_000, 9)])
    rng.shuffle(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    keys = _keys(int(off[-1]), 51)
    Ps = rng.choice([1024, 2500, 4096], size=sizes.size).astype(np.uint32)
    prm = ph.make_params(7.0, alpha, 2500, seed=3, encoder=enc, keep_pilots=True,
                         warps_per_partition=2 if enc else 1,
                         search_schedule=2 if enc % 2 == 0 else 1)  # the work queue, and one CTA per partition
    hs = ph.phobic_build_batch(_dev(keys), off, prm, partition_sizes=Ps)
    assert len(hs) == sizes.size
    for s, h in enumerate(hs):
        ks = keys[off[s]:off[s + 1]]
        o = orc.Oracle(ks, lam=7.0, alpha=alpha, P=int(Ps[s]), encoder=enc, seed=3, threads=0)
        assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots), s
        compare_structure(ph, o, h, enc)
        got = _host(h.query(_dev(ks)))
        assert np.array_equal(got, o.query(ks)), s
    # handles share one allocation: free in an arbitrary order, the rest stay valid
    last = hs[-1]
    for h in hs[:-1]:
        h.free()
    ks = keys[off[-2]:off[-1]]
    assert np.array_equal(np.sort(_host(last.query(_dev(ks)))), np.arange(ks.size, dtype=np.uint64))
