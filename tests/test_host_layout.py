"""Host-side layout of packed dictionaries (mrom_rom_from_packed's input), checked without a GPU:
16-byte aligned regions inside the buffer, in the documented order, holding the arrays exactly."""
import numpy as np

from workloads import reduced_object


def test_packed_dictionary_layout():
    import paper_2307_05590_gb300 as m
    objs = [reduced_object(20230711, 40 + k, r) for k, r in enumerate([3, 7, 12, 5])]
    items = []
    for k, o in enumerate(objs):
        it = dict(r=o.r, K=o.K, C=o.C, B=o.B, c00=o.c00, alpha=o.alpha, alpha_lb=o.alpha_lb, vol_B=o.vol_B)
        if k % 2 == 0:
            it["G"] = o.G
        if k != 2:
            it["K_in"] = o.K_in
        if k == 3:
            it["Me"] = 1e-3 * np.eye(o.r, dtype=np.complex128)
            it["N0"] = np.arange(9.0).reshape(3, 3)
        items.append(it)
    pk = m.PackedDictionary(items, pin=False)
    buf = np.asarray(pk.buffer)
    end = 0
    for e, it in zip(pk.entries, items):
        r = it["r"]
        assert e.offset % 16 == 0 and e.offset >= end
        names = ["K"] + (["K_in"] if "K_in" in it else []) + ["C"] + (["Me"] if "Me" in it else []) + ["B"] \
            + (["G"] if "G" in it else [])
        pos = e.offset
        for nm in names:
            a = np.ascontiguousarray(it[nm], dtype=np.complex128)
            got = np.frombuffer(buf[pos:pos + a.nbytes].tobytes(), dtype=np.complex128).reshape(a.shape)
            assert np.array_equal(got, a), nm
            pos += a.nbytes
        end = pos
        assert (e.has_kin, e.has_me, e.has_gram) == ("K_in" in it, "Me" in it, "G" in it)
        assert np.array_equal(np.array(e.c00[:]), np.asarray(it["c00"]).ravel())
        assert np.array_equal(np.array(e.N0[:]), np.asarray(it.get("N0", np.zeros(9))).ravel())
        assert e.r == r
    assert end <= pk.nbytes and pk.nbytes % 16 == 0
