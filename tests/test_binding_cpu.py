"""The ctypes binding's argument marshalling, without a GPU: inputs are
converted on the host or passed through as tensors of the declared dtype, and
output buffers are filled in place, so a buffer of the wrong type, layout or
size is refused before the library could write past it or into a copy."""
import ctypes as ct

import numpy as np
import pytest

from paper_1307_8052_gb300 import binding as b

torch = pytest.importorskip("torch")


def test_inputs_convert_on_the_host_and_tensors_keep_their_dtype():
    keep = []
    p = b._ptr([1, 2, 3], np.int32, keep)
    assert keep[-1].dtype == np.int32 and p.value == keep[-1].ctypes.data
    a = np.arange(6.0)
    assert b._ptr(a, np.float64, keep).value == a.ctypes.data   # no copy when nothing changes
    t = torch.zeros(4, dtype=torch.complex128)
    assert b._ptr(t, np.complex128).value == t.data_ptr()
    with pytest.raises(TypeError):
        b._ptr(torch.zeros(4, dtype=torch.complex64), np.complex128)
    with pytest.raises(TypeError):
        b._ptr(torch.zeros(4, dtype=torch.int64), np.int32)
    with pytest.raises(ValueError):
        b._ptr(torch.zeros((4, 4), dtype=torch.complex128).t(), np.complex128)


def test_outputs_are_written_in_place_or_refused():
    good = np.zeros((2, 3), dtype=np.complex128)
    assert b._out_ptr(good, np.complex128, 6).value == good.ctypes.data
    assert b._out_ptr(good, np.complex128).value == good.ctypes.data
    bad = [np.zeros((2, 3), dtype=np.complex64),            # narrower: the library would write past it
           np.zeros((3, 2), dtype=np.complex128).T,          # not C-contiguous: a copy would be filled
           np.zeros((2, 2), dtype=np.complex128),            # too small
           [0j] * 6]                                         # not an array
    ro = np.zeros((2, 3), dtype=np.complex128)
    ro.flags.writeable = False
    bad.append(ro)
    for x in bad:
        with pytest.raises(ValueError):
            b._out_ptr(x, np.complex128, 6)
    t = torch.zeros((2, 3), dtype=torch.complex128)
    assert b._out_ptr(t, np.complex128, 6).value == t.data_ptr()
    for x in (torch.zeros(6, dtype=torch.complex64), torch.zeros((3, 2), dtype=torch.complex128).t(),
              torch.zeros(5, dtype=torch.complex128)):
        with pytest.raises(ValueError):
            b._out_ptr(x, np.complex128, 6)


class _FakeLib:
    """Records the calls of the wrappers; rpa_gvectors reports NG = 3."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append((name, args))
            if name == "rpa_gvectors":
                ct.cast(args[2], ct.POINTER(ct.c_int32))[0] = 3
            return b.RPA_OK
        return fn


def test_wrappers_pass_the_caller_buffers(monkeypatch):
    fake = _FakeLib()
    monkeypatch.setattr(b, "_lib", fake)
    om = np.array([0.5, 1.0])
    out = b.rpa_chi0("ctx", 0, om)
    assert out.shape == (2, 3, 3) and out.dtype == np.complex128
    name, args = fake.calls[-1]
    assert name == "rpa_chi0" and args[4].value == out.ctypes.data
    mine = np.zeros((2, 3, 3), dtype=np.complex128)
    assert b.rpa_epsilon_inv("ctx", 0, om, mine) is mine
    assert fake.calls[-1][1][4].value == mine.ctypes.data
    with pytest.raises(ValueError):
        b.rpa_chi0("ctx", 0, om, np.zeros((2, 3, 3), dtype=np.complex64))
    with pytest.raises(ValueError):
        b.rpa_chi0("ctx", 0, om, np.zeros((1, 3, 3), dtype=np.complex128))
    # gradient outputs: one pointer per set and q-point, in place, NULL for None
    dC = [np.zeros((2, 5), dtype=np.complex128), None]
    dchi = [np.zeros((2, 3, 3), dtype=np.complex128)]
    b.rpa_energy_backward("ctx", [0], [1.0], om, [1.0, 1.0], 1.0, [0, 1], dC, None, dchi)
    name, args = fake.calls[-1]
    assert name == "rpa_energy_backward"
    ptrs = ct.cast(args[11], ct.POINTER(ct.c_void_p))
    assert ptrs[0] == dC[0].ctypes.data and ptrs[1] is None and args[12] is None
    assert ct.cast(args[13], ct.POINTER(ct.c_void_p))[0] == dchi[0].ctypes.data
    with pytest.raises(ValueError):
        b.rpa_energy_backward("ctx", [0], [1.0], om, [1.0, 1.0], 1.0, [0], [np.zeros(4, dtype=np.complex64)])
    with pytest.raises(ValueError):
        b.rpa_energy_backward("ctx", [0], [1.0], om, [1.0, 1.0], 1.0, [0], None, None,
                              [np.zeros((2, 2, 2), dtype=np.complex128)])


def test_host_arrays_must_match_the_sizes_the_library_reads(monkeypatch):
    fake = _FakeLib()
    monkeypatch.setattr(b, "_lib", fake)
    C = np.zeros((4, 6), dtype=np.complex128)
    mil = np.zeros((6, 3), dtype=np.int32)
    b.rpa_set_orbitals("ctx", 0, [0.0, 0.0, 0.0], mil, C, np.zeros(4), np.ones(4))
    assert fake.calls[-1][0] == "rpa_set_orbitals"
    for bad in ({"miller": mil[:5]}, {"eps": np.zeros(3)}, {"f": np.ones(5)}, {"k_red": [0.0, 0.0]}):
        kw = dict(k_red=[0.0, 0.0, 0.0], miller=mil, eps=np.zeros(4), f=np.ones(4))
        kw.update(bad)
        with pytest.raises(ValueError):
            b.rpa_set_orbitals("ctx", 0, kw["k_red"], kw["miller"], C, kw["eps"], kw["f"])
    b.rpa_set_qpoint("ctx", 0, [0.5, 0, 0], [0, 1], [1, 0], [[0, 0, 0], [1, 0, 0]])
    with pytest.raises(ValueError):
        b.rpa_set_qpoint("ctx", 0, [0.5, 0, 0], [0, 1], [1], [[0, 0, 0], [1, 0, 0]])
    with pytest.raises(ValueError):
        b.rpa_set_qpoint("ctx", 0, [0.5, 0, 0], [0, 1], [1, 0], [[0, 0, 0]])
    om = np.array([0.5, 1.0])
    b.rpa_energy("ctx", [0, 1], [0.5, 0.5], om, [1.0, 1.0])
    with pytest.raises(ValueError):
        b.rpa_energy("ctx", [0, 1], [1.0], om, [1.0, 1.0])
    with pytest.raises(ValueError):
        b.rpa_energy("ctx", [0], [1.0], om, [1.0])
    with pytest.raises(ValueError):
        b.rpa_energy_collect("ctx", [1.0], [1.0, 1.0], 2)
