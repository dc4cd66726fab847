"""Host-side checks of libmt that need no GPU: the library loads, exports
every function include/mt.h declares, and resolves / validates parameters
(grid bits, default cutoff, cell width, workspace size) without touching a
device."""
import re
from pathlib import Path

import numpy as np
import pytest

from paper_1811_05474_gb300 import mt

HEADER = Path(__file__).resolve().parents[1] / "include" / "mt.h"


def declared():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mt_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    L = mt.lib()
    names = declared()
    assert "mt_create" in names and "mt_step" in names and "mt_run" in names
    assert "mt_read_masses" in names
    for name in names:
        assert hasattr(L, name), name


def test_binding_wraps_every_declared_function():
    for name in declared():
        assert hasattr(mt, name), name


def test_defaults_and_default_cutoff():
    p = mt.mt_params_init()
    assert p.dim == 1 and p.D_mt == 0.1 and p.dt == 1.0 and p.react == 1
    r = mt.mt_resolve(p)
    assert r.cutoff == pytest.approx(3 * np.sqrt(4 * 0.1 * 1.0), rel=1e-15)


def test_frac_bits_rule():
    # largest k with s_max 2^k < 2^30 and L 2^k < 2^61
    for L, D in ((1000.0, 0.1), (1e6, 0.1), (50.0, 0.5), (1e9, 0.1), (3.0, 10.0)):
        r = mt.mt_resolve(mt.mt_params_init(n=10, L=(L,), D_mt=D))
        k = r.frac_bits
        assert r.cutoff * 2.0 ** k < 2 ** 30 and L * 2.0 ** k < 2 ** 61
        assert r.cutoff * 2.0 ** (k + 1) >= 2 ** 30 or L * 2.0 ** (k + 1) >= 2 ** 61


def test_cell_width_rules():
    # 1-d: about two particles per sort cell
    r = mt.mt_resolve(mt.mt_params_init(n=10 ** 6, L=(1e6,)))
    width = 2.0 ** r.cell_shift * 2.0 ** -r.frac_bits
    assert 1.0 <= width <= 4.0
    # 2-d: cells wider than the cutoff
    r2 = mt.mt_resolve(mt.mt_params_init(dim=2, n=1000, L=(100.0, 100.0)))
    assert 2.0 ** r2.cell_shift > np.floor(r2.cutoff * 2.0 ** r2.frac_bits)


@pytest.mark.parametrize("field,value", [
    ("dim", 3), ("n", -1), ("D_mt", 0.0), ("dt", -1.0), ("D_rw", -0.1),
    ("search", 7), ("precision", 4), ("norm", 9), ("react", 2), ("observe_cap", -5),
    ("frac_bits", 63),
])
def test_invalid_parameters_rejected(field, value):
    p = mt.mt_params_init(n=10)
    setattr(p, field, value)
    with pytest.raises(mt.MtError) as e:
        mt.mt_resolve(p)
    assert e.value.status == mt.MT_ERR_INVALID
    assert mt.mt_last_error()


def test_invalid_domain_rejected():
    with pytest.raises(mt.MtError):
        mt.mt_resolve(mt.mt_params_init(n=10, L=(0.0,)))
    with pytest.raises(mt.MtError):
        mt.mt_resolve(mt.mt_params_init(n=10, L=(float("inf"),)))
    with pytest.raises(mt.MtError):  # grid would overflow 61 bits
        mt.mt_resolve(mt.mt_params_init(n=10, L=(1e6,), frac_bits=60))


def test_workspace_grows_with_n_and_observables():
    b1 = mt.mt_workspace_bytes(mt.mt_params_init(n=1000))
    b2 = mt.mt_workspace_bytes(mt.mt_params_init(n=2000))
    b3 = mt.mt_workspace_bytes(mt.mt_params_init(n=1000, observe_cap=100))
    assert b2 > b1 and b3 >= b1 + 100 * 32
    # algorithmic state (x, A, B double buffered) is a lower bound
    assert b1 >= 2 * 1000 * 24


def test_create_rejects_missing_workspace():
    p = mt.mt_params_init(n=10)
    with pytest.raises(mt.MtError) as e:
        mt.mt_create(p, None, 0, None)
    assert e.value.status == mt.MT_ERR_WORKSPACE


def test_philox_reference_matches_published_kat():
    from tests.philox_ref import philox4x32_10, load_kat

    for ctr, key, out in load_kat():
        assert philox4x32_10(ctr, key) == out


def _batch_params(**kw):
    return mt.mt_params_init(dim=1, L=(1.0,), **kw)


def test_batch_resolve_lays_realisations_side_by_side():
    ns, Ls = [1000, 10, 250000], [1000.0, 3.5, 2.5e5]
    b = mt.make_batch(ns, Ls)
    r = mt.mt_batch_resolve(_batch_params(), b)
    assert r.n == sum(ns)
    assert r.frac_bits == mt.mt_resolve(mt.mt_params_init(n=ns[2], L=(Ls[2],))).frac_bits
    # the shared axis holds every domain plus gaps wider than the cutoff
    w = 2.0 ** (r.cell_shift - r.frac_bits)
    assert r.L[0] >= sum(Ls) + 2 * r.cutoff
    assert r.L[0] <= sum(Ls) + len(ns) * (2 * r.cutoff + 3 * w)
    assert 16 <= r.seg_target <= 1024
    single = mt.mt_workspace_bytes(mt.mt_params_init(n=sum(ns), L=(r.L[0],)))
    assert mt.mt_batch_workspace_bytes(_batch_params(), b) >= single // 2
    # a batch of one is a single system
    one = mt.mt_batch_resolve(_batch_params(), mt.make_batch([5000], [5000.0]))
    ref = mt.mt_resolve(mt.mt_params_init(n=5000, L=(5000.0,)))
    assert (one.n, one.frac_bits, one.cell_shift, one.seg_target) == \
        (ref.n, ref.frac_bits, ref.cell_shift, ref.seg_target)
    assert one.L[0] >= 5000.0


def test_batch_rejects_bad_descriptions():
    p = _batch_params()
    for ns, Ls in (([10, 0], [10.0, 10.0]), ([10], [-1.0]), ([], []), ([10], [float("nan")])):
        with pytest.raises(mt.MtError) as e:
            mt.mt_batch_resolve(p, mt.make_batch(ns, Ls))
        assert e.value.status == mt.MT_ERR_INVALID
    with pytest.raises(mt.MtError):
        mt.mt_batch_resolve(mt.mt_params_init(dim=2, L=(10.0, 10.0)), mt.make_batch([10], [10.0]))
    with pytest.raises(mt.MtError):
        mt.mt_batch_resolve(_batch_params(search=mt.MT_SEARCH_BRUTE), mt.make_batch([10], [10.0]))
    # realisation index bits: 2^20 particles leave room for 2^11 realisations
    with pytest.raises(mt.MtError):
        mt.mt_batch_resolve(p, mt.make_batch([2 ** 20] + [1] * 2048, [1e6] + [1.0] * 2048))


def test_seg_target_is_validated_and_kept():
    r = mt.mt_resolve(mt.mt_params_init(n=100000, L=(1e5,), seg_target=256))
    assert r.seg_target == 256
    with pytest.raises(mt.MtError):
        mt.mt_resolve(mt.mt_params_init(n=100000, L=(1e5,), seg_target=8))
    # no one-kernel step for 2-d or brute force
    assert mt.mt_resolve(mt.mt_params_init(dim=2, n=100, L=(10.0, 10.0))).seg_target == 0


def test_periodic_walls_rules():
    r = mt.mt_resolve(mt.mt_params_init(n=1000, L=(1000.0,), walls=mt.MT_WALLS_PERIODIC))
    assert r.walls == mt.MT_WALLS_PERIODIC and r.seg_target == 0  # general pipeline
    mt.mt_resolve(mt.mt_params_init(dim=2, n=100, L=(10.0, 10.0), walls=mt.MT_WALLS_PERIODIC))
    for bad in (dict(dim=2, n=100, L=(10.0, 3.0)),                  # cutoff >= L[1] / 2
                dict(n=10, L=(3.0,)),                                # cutoff >= L / 2
                dict(n=10, L=(100.0,), search=mt.MT_SEARCH_BRUTE, cutoff=60.0),
                dict(n=10, L=(100.0,), walls=7)):
        kw = dict(walls=mt.MT_WALLS_PERIODIC)
        kw.update(bad)
        with pytest.raises(mt.MtError) as e:
            mt.mt_resolve(mt.mt_params_init(**kw))
        assert e.value.status == mt.MT_ERR_INVALID
    mt.mt_resolve(mt.mt_params_init(dim=2, n=100, L=(10.0, 10.0), search=mt.MT_SEARCH_BRUTE,
                                    walls=mt.MT_WALLS_PERIODIC))
    # batches: each realisation wraps on its own domain, which must exceed 2 s_max
    rb = mt.mt_batch_resolve(mt.mt_params_init(dim=1, L=(1.0,), walls=mt.MT_WALLS_PERIODIC),
                             mt.make_batch([10, 20], [10.0, 20.0]))
    assert rb.walls == mt.MT_WALLS_PERIODIC and rb.seg_target == 0
    with pytest.raises(mt.MtError):
        mt.mt_batch_resolve(mt.mt_params_init(dim=1, L=(1.0,), walls=mt.MT_WALLS_PERIODIC),
                            mt.make_batch([10, 20], [10.0, 3.0]))


def test_species_rules():
    r = mt.mt_resolve(mt.mt_params_init(n=1000, L=(1000.0,)))
    assert r.species == 2 and r.seg_target > 0  # default: A and B, one-kernel step
    r4 = mt.mt_resolve(mt.mt_params_init(n=1000, L=(1000.0,), species=4))
    assert r4.species == 4 and r4.seg_target == 0  # multi-kernel pipeline
    w3 = mt.mt_workspace_bytes(mt.mt_params_init(n=10000, L=(1e4,), species=3))
    w6 = mt.mt_workspace_bytes(mt.mt_params_init(n=10000, L=(1e4,), species=6))
    assert abs((w6 - w3) - 2 * 3 * 10000 * 8) <= 512  # two buffers, three more species
    mt.mt_resolve(mt.mt_params_init(n=10, species=mt.MT_MAX_SPECIES))
    for bad in (dict(species=1), dict(species=mt.MT_MAX_SPECIES + 1), dict(species=-2),
                dict(stored_p=-1)):
        with pytest.raises(mt.MtError) as e:
            mt.mt_resolve(mt.mt_params_init(n=10, **bad))
        assert e.value.status == mt.MT_ERR_INVALID
    # a batch with more species runs the multi-kernel pipeline
    rb = mt.mt_batch_resolve(_batch_params(species=3), mt.make_batch([100, 50], [100.0, 50.0]))
    assert rb.species == 3 and rb.seg_target == 0


def test_stored_p_rules():
    # the band follows the mean density: 1.9 right neighbours per particle here
    r = mt.mt_resolve(mt.mt_params_init(n=100000, L=(1e5,), stored_p=1))
    assert 8 <= r.stored_p <= 32 and r.seg_target == 0
    dense = mt.mt_resolve(mt.mt_params_init(n=100000, L=(500.0,), D_mt=0.5, dt=0.1, stored_p=1))
    mean = dense.cutoff * 100000 / 500.0
    assert mean * 1.2 <= dense.stored_p <= mean * 1.6 + 16
    assert mt.mt_resolve(mt.mt_params_init(n=1000, L=(1e3,), stored_p=40)).stored_p == 40
    assert mt.mt_resolve(mt.mt_params_init(n=10, L=(1e3,), stored_p=40)).stored_p == 10
    base = mt.mt_workspace_bytes(mt.mt_params_init(n=10000, L=(1e4,), stored_p=0, species=3))
    w = mt.mt_workspace_bytes(mt.mt_params_init(n=10000, L=(1e4,), stored_p=20, species=3))
    assert abs((w - base) - (2 * 10000 * 4 + 20 * 10016 * 8)) <= 512  # counts + FP64 band
    for bad in (dict(dim=2, L=(10.0, 10.0)), dict(search=mt.MT_SEARCH_BRUTE),
                dict(search=mt.MT_SEARCH_FULL)):
        with pytest.raises(mt.MtError) as e:
            mt.mt_resolve(mt.mt_params_init(n=10, stored_p=1, **bad))
        assert e.value.status == mt.MT_ERR_INVALID
    assert mt.mt_batch_resolve(_batch_params(stored_p=1), mt.make_batch([10], [10.0])).stored_p >= 2


def test_checkpoint_params_rejects_foreign_files(tmp_path):
    with pytest.raises(mt.MtError) as e:
        mt.mt_checkpoint_params(tmp_path / "missing.ckpt")
    assert e.value.status == mt.MT_ERR_INVALID
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"not a checkpoint" * 20)
    with pytest.raises(mt.MtError) as e:
        mt.mt_checkpoint_params(junk)
    assert e.value.status == mt.MT_ERR_INVALID
