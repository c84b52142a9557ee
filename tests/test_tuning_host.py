"""The tuner's host side without a GPU: candidate lists, the geometry key, the JSON cache (the counterpart of
the guide's FFTW wisdom file, digHoloFFTWWisdomFilename) and validation of explicit tunings."""
import json

import pytest

import paper_2204_02348_gb300 as dh
from synth import holograms as syn

FUSED, PRUNED, GENERIC, GROUPS = (dh.DH_VARIANT_FUSED, dh.DH_VARIANT_FUSED_PRUNED, dh.DH_VARIANT_GENERIC,
                                  dh.DH_VARIANT_FUSED_GROUPS)


@pytest.fixture()
def handle():
    h = dh.dh_create()
    yield h
    dh.dh_destroy(h)


def test_candidates_for_the_batching_geometry(handle):
    dh.configure(handle, syn.setup_batching())
    c = dh.dh_tuning_candidates(handle)
    assert [x["variant"] for x in c] == [GROUPS, FUSED, PRUNED, GENERIC]
    assert all(x["chunk_mb"] == 0 and x["radix"] == [] for x in c)
    # the split-BF16 overlap has neither the pruned nor the group variant
    dh.dh_set_precision(handle, dh.DH_PRECISION_SPLIT_BF16)
    assert [x["variant"] for x in dh.dh_tuning_candidates(handle)] == [FUSED, GENERIC]


def test_candidates_for_the_precision_geometry(handle):
    dh.configure(handle, syn.setup_precision())
    c = dh.dh_tuning_candidates(handle)
    plans = [[8, 4, 3], [3, 4, 8], [4, 8, 3], [16, 2, 3]]
    # the 256 x 256 fused kernel first, then the generic path's chunk sizes and radix plans
    expect = [{"variant": FUSED, "chunk_mb": 0, "radix": []}]
    expect += [{"variant": GENERIC, "chunk_mb": mb, "radix": p} for mb in (24, 48, 96) for p in plans]
    assert c == expect
    # the split-BF16 overlap has the same candidates (the fused kernel's tensor-core variant first)
    dh.dh_set_precision(handle, dh.DH_PRECISION_SPLIT_BF16)
    assert dh.dh_tuning_candidates(handle) == expect
    dh.dh_set_precision(handle, dh.DH_PRECISION_FP32)
    for x in c[1:]:
        prod = 1
        for r in x["radix"]:
            prod *= r
        assert prod == 96
    assert dh.dh_tuning_candidates(handle) == c   # deterministic


def test_key_names_the_geometry(handle):
    s = syn.setup_precision()
    dh.configure(handle, s)
    assert dh.dh_tuning_key(handle) == f"N256_M96_G15_P2_W{s.frame_w}_H{s.frame_h}_prec0_basis0"
    dh.dh_set_precision(handle, dh.DH_PRECISION_SPLIT_BF16)
    assert dh.dh_tuning_key(handle).endswith("_prec1_basis0")


def test_cache_round_trip_and_explicit_tuning(handle, tmp_path):
    s = syn.setup_precision()
    dh.configure(handle, s)
    key = dh.dh_tuning_key(handle)
    assert dh.dh_get_tuning(handle) == {"variant": 0, "chunk_mb": 0, "radix": []}
    path = tmp_path / "tuning.json"
    path.write_text(json.dumps({"format": "digholo-gb300-tuning", "version": 1, "entries": [
        {"key": key, "variant": GENERIC, "chunk_mb": 96, "radix": [4, 8, 3], "ms": 0.5},
        {"key": "N128_M64_G9_P2_W320_H256_prec0_basis0", "variant": FUSED, "chunk_mb": 0, "radix": []}]}))
    dh.dh_set_tuning_cache(handle, str(path))
    assert dh.dh_get_tuning(handle) == {"variant": GENERIC, "chunk_mb": 96, "radix": [4, 8, 3]}
    # an explicit tuning wins for this key; None goes back to the cache
    dh.dh_set_tuning(handle, {"variant": GENERIC, "chunk_mb": 24, "radix": [16, 2, 3]})
    assert dh.dh_get_tuning(handle) == {"variant": GENERIC, "chunk_mb": 24, "radix": [16, 2, 3]}
    dh.dh_set_tuning(handle, None)
    assert dh.dh_get_tuning(handle)["chunk_mb"] == 96
    # another geometry finds its own entry
    dh.configure(handle, syn.setup_batching())
    assert dh.dh_get_tuning(handle) == {"variant": FUSED, "chunk_mb": 0, "radix": []}
    dh.dh_set_tuning_cache(handle, None)
    assert dh.dh_get_tuning(handle) == {"variant": 0, "chunk_mb": 0, "radix": []}


def test_missing_cache_is_empty_and_malformed_cache_is_rejected(handle, tmp_path):
    dh.configure(handle, syn.setup_precision())
    dh.dh_set_tuning_cache(handle, str(tmp_path / "absent.json"))
    assert dh.dh_get_tuning(handle)["variant"] == 0
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"format": "digholo-gb300-tuning", "version": 1, "entries": [
        {"key": dh.dh_tuning_key(handle), "variant": GENERIC, "chunk_mb": 48, "radix": [8, 4, 3]}]}))
    dh.dh_set_tuning_cache(handle, str(good))
    for bad in ('{"format": "digholo-gb300-tuning", "entries": [', '{"format": "other", "entries": []}',
                '{"format": "digholo-gb300-tuning", "entries": [{"key": "k", "variant": 9, "chunk_mb": 0}]}',
                '{"format": "digholo-gb300-tuning", "entries": [{"key": "k", "variant": 3, "chunk_mb": 0, '
                '"radix": [6]}]}', '[] trailing'):
        p = tmp_path / "bad.json"
        p.write_text(bad)
        with pytest.raises(dh.DigHoloError) as e:
            dh.dh_set_tuning_cache(handle, str(p))
        assert e.value.code == dh.DH_ERROR_INVALIDARGUMENT
    # the good cache loaded before is still in effect
    assert dh.dh_get_tuning(handle)["chunk_mb"] == 48


def test_invalid_tunings_rejected(handle):
    dh.configure(handle, syn.setup_precision())
    for t in ({"variant": 7}, {"variant": GENERIC, "chunk_mb": -1}, {"variant": GENERIC, "radix": [8, 4, 4]},
              {"variant": GENERIC, "radix": [6, 16]}, {"variant": GENERIC, "radix": [2] * 7}):
        with pytest.raises((dh.DigHoloError, IndexError)):
            dh.dh_set_tuning(handle, t)
    assert dh.dh_get_tuning(handle)["variant"] == 0
