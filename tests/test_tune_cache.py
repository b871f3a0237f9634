"""The autotuner's cache (host logic, no GPU): entries are recorded, looked
up, listed in key order, persisted to a text file and loaded back, and a
malformed file or key is refused.  What the tuner times is covered on the GPU
by every test that runs the tuned kernels (their candidates give identical
results, so the parity tests hold whatever it picks)."""
import os

import pytest


@pytest.fixture()
def afn(tmp_path):
    from paper_2304_05460_gb300 import afn as a
    a.afn_tune_set_cache(None)
    a.afn_tune_clear()
    yield a
    a.afn_tune_set_cache(None)
    a.afn_tune_clear()


def test_put_get_list_clear(afn):
    afn.afn_tune_put("mv32u/ds8/nb4/ker0/n2^15/sm103x152", 1)
    afn.afn_tune_put("fsai/wm64/f32/k2^11/nr2^15/sm103x152", 0)
    afn.afn_tune_put("mv32u/ds8/nb4/ker0/n2^15/sm103x152", 0)      # overwrite
    assert afn.afn_tune_get("mv32u/ds8/nb4/ker0/n2^15/sm103x152") == 0
    ent = afn.afn_tune_entries()
    assert ent == {"fsai/wm64/f32/k2^11/nr2^15/sm103x152": 0,
                   "mv32u/ds8/nb4/ker0/n2^15/sm103x152": 0}
    assert list(ent) == sorted(ent)
    with pytest.raises(afn.AfnError) as e:
        afn.afn_tune_get("gmv32/tiles2^9/sm103x152")
    assert e.value.status == afn.AFN_ERR_ARG
    afn.afn_tune_clear()
    assert afn.afn_tune_entries() == {}


def test_bad_keys_and_choices_refused(afn):
    for key, ch in (("has space", 1), ("", 1), ("x" * 201, 1), ("ok/key", -1)):
        with pytest.raises(afn.AfnError):
            afn.afn_tune_put(key, ch)
    assert afn.afn_tune_entries() == {}


def test_persisted_round_trip(afn, tmp_path):
    path = tmp_path / "tune.txt"
    afn.afn_tune_set_cache(path)                 # a new file is created
    afn.afn_tune_put("gmv32/tiles2^9/sm103x152", 2)
    afn.afn_tune_put("gapply/tiles2^12/sm103x152", 1)
    lines = [l for l in path.read_text().splitlines() if not l.startswith("#")]
    assert sorted(lines) == ["gapply/tiles2^12/sm103x152 1", "gmv32/tiles2^9/sm103x152 2"]
    # a fresh process state: forget, then load the file back
    afn.afn_tune_set_cache(None)
    afn.afn_tune_clear()
    assert afn.afn_tune_entries() == {}
    afn.afn_tune_set_cache(path)
    assert afn.afn_tune_entries() == {"gapply/tiles2^12/sm103x152": 1,
                                      "gmv32/tiles2^9/sm103x152": 2}
    # entries in memory survive loading a file that lacks them, and are written back
    afn.afn_tune_set_cache(None)
    afn.afn_tune_put("fsai/wm32/f64/k2^8/nr2^11/sm103x152", 1)
    afn.afn_tune_set_cache(path)
    assert len(afn.afn_tune_entries()) == 3
    assert "fsai/wm32/f64/k2^8/nr2^11/sm103x152 1" in path.read_text()


def test_malformed_cache_refused(afn, tmp_path):
    bad = tmp_path / "bad.txt"
    bad.write_text("# afn autotuner cache v1: key choice\nkey-without-choice\n")
    with pytest.raises(afn.AfnError) as e:
        afn.afn_tune_set_cache(bad)
    assert e.value.status == afn.AFN_ERR_ARG
    neg = tmp_path / "neg.txt"
    neg.write_text("a/b -3\n")
    with pytest.raises(afn.AfnError):
        afn.afn_tune_set_cache(neg)
    with pytest.raises(afn.AfnError):
        afn.afn_tune_set_cache(tmp_path / "no_such_dir" / "x.txt")
