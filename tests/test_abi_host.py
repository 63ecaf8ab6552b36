"""C ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/elsr.h, and rejects invalid instances in its
host-side validation (before any device call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1704_05132_gb300 import _native as nat
from paper_1704_05132_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return nat.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "elsr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(elsr_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("elsr_create", "elsr_eval_neighbourhood", "elsr_vns_run", "elsr_result",
              "elsr_destroy", "elsr_batch_run", "elsr_multistart_run"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) == set(nat.SIGNATURES)


def test_version_and_strerror(lib):
    assert lib.elsr_version() >= 10000
    assert lib.elsr_strerror(nat.ELSR_E_RANGE)


def _create(lib, K, T, D, R, c):
    h = ctypes.c_void_p()
    arrs = [np.ascontiguousarray(a, np.int32) for a in (D, R, c[0], c[1], c[2], c[3])]
    code = lib.elsr_create(ctypes.byref(h), K, T, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs])
    return code, h


def test_validation_rejects_bad_instances(lib):
    K, T = 2, 4
    D = np.ones((K, T))
    R = np.zeros((K, T))
    c = [np.ones(K)] * 4
    assert _create(lib, K, 0, D, R, c)[0] == nat.ELSR_E_ARG
    assert _create(lib, K, 129, np.ones((K, 129)), np.zeros((K, 129)), c)[0] == nat.ELSR_E_ARG
    assert _create(lib, 0, T, D, R, c)[0] == nat.ELSR_E_ARG
    Dn = D.copy()
    Dn[1, 2] = -1
    code, h = _create(lib, K, T, Dn, R, c)
    assert code == nat.ELSR_E_ARG and not h.value
    assert b"negative" in lib.elsr_last_error(None)
    big = np.full((K, T), 2**30)
    assert _create(lib, K, T, big, R, c)[0] == nat.ELSR_E_RANGE
    hm = [np.ones(K), np.ones(K), np.full(K, 2**30), np.ones(K)]
    assert _create(lib, K, T, np.full((K, T), 1000), R, hm)[0] == nat.ELSR_E_RANGE


def test_checkpoint_struct_and_file_roundtrip(tmp_path):
    """elsr_checkpoint_t as the binding lays it out (96 bytes: six 32-bit and
    nine 64-bit fields), and a checkpoint survives an .npz round trip with
    full 64-bit seed and hash values."""
    from paper_1704_05132_gb300 import elsr
    assert ctypes.sizeof(nat.Checkpoint) == 96
    ck = {n: i + 1 for i, (n, _) in enumerate(nat.Checkpoint._fields_)}
    ck["seed"] = (1 << 64) - 3
    ck["traj_hash"] = 0x9E3779B97F4A7C15
    ck["gM"] = np.eye(3, 5, dtype=np.uint8)
    ck["gR"] = np.ones((3, 5), np.uint8)
    path = str(tmp_path / "ck.npz")
    elsr.save_checkpoint(path, ck)
    back = elsr.load_checkpoint(path)
    for n, _ in nat.Checkpoint._fields_:
        assert back[n] == ck[n], n
    assert (back["gM"] == ck["gM"]).all() and (back["gR"] == ck["gR"]).all()
    c = nat.Checkpoint.from_dict(back)
    assert c.seed == ck["seed"] and c.traj_hash == ck["traj_hash"]


def _create_ex(lib, K, T, D, R, c, pm, pr):
    h = ctypes.c_void_p()
    arrs = [np.ascontiguousarray(a, np.int32) for a in (D, R, c[0], c[1], c[2], c[3])]
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
    pms = None if pm is None else np.ascontiguousarray(pm, np.int32)
    prs = None if pr is None else np.ascontiguousarray(pr, np.int32)
    code = lib.elsr_create_ex(ctypes.byref(h), K, T, *[p(a) for a in arrs], p(pms), p(prs))
    return code, h


def test_production_costs_validated_on_the_host(lib):
    """Unit production costs: negative values, values from 2^24 on, and one
    array without the other are refused before any device work."""
    K, T = 3, 5
    D = np.full((K, T), 7)
    R = np.zeros((K, T))
    c = [np.full(K, 100), np.full(K, 50), np.full(K, 2), np.full(K, 1)]
    assert _create_ex(lib, K, T, D, R, c, [1, -1, 0], [0, 0, 0])[0] == nat.ELSR_E_ARG
    assert _create_ex(lib, K, T, D, R, c, [0, 0, 0], [0, 1 << 24, 0])[0] == nat.ELSR_E_RANGE
    code, h = _create_ex(lib, K, T, D, R, c, [1, 2, 3], None)
    assert code == nat.ELSR_E_ARG and not h.value
    assert b"pM and pR" in lib.elsr_last_error(None)


def test_new_entry_points_reject_a_null_handle(lib):
    """Fork-join, time budget, checkpoint, resume and the staging pass return
    ELSR_E_ARG for a NULL handle (and touch nothing)."""
    ck = nat.Checkpoint()
    gm = np.zeros(4, np.uint8)
    P = ctypes.c_void_p
    assert lib.elsr_vns_forkjoin_run(None, 0, 10, 3, 0, 2) == nat.ELSR_E_ARG
    assert lib.elsr_set_time_limit(None, 1000) == nat.ELSR_E_ARG
    assert lib.elsr_checkpoint(None, ctypes.byref(ck), None, None) == nat.ELSR_E_ARG
    assert lib.elsr_vns_resume(None, ctypes.byref(ck), gm.ctypes.data_as(P),
                               gm.ctypes.data_as(P), 5) == nat.ELSR_E_ARG
    assert lib.elsr_batch_stage_tables(None) == nat.ELSR_E_ARG


def test_empty_batch_refused_before_any_call():
    """A batch of no instances is refused by the binding with a clear error,
    before the library is asked for anything."""
    from paper_1704_05132_gb300 import elsr
    with pytest.raises(ValueError, match="at least one instance"):
        elsr.Batch([])


def test_binding_checks_array_shapes_before_the_library_reads_them():
    """The library reads K*T and K entries behind the pointers it is given;
    the binding refuses arrays of other shapes instead of passing them on."""
    from paper_1704_05132_gb300 import elsr, gen
    g = gen.make_instance(1, 1, K=4, T=6)
    bad = [
        gen.ElsrInstance(g.D, g.R[:, :5], g.kM, g.kR, g.hM, g.hR),          # R shorter
        gen.ElsrInstance(g.D[0], g.R[0], g.kM, g.kR, g.hM, g.hR),           # 1-D rows
        gen.ElsrInstance(g.D, g.R, g.kM[:3], g.kR, g.hM, g.hR),             # kM too short
        gen.ElsrInstance(g.D, g.R, g.kM, g.kR, g.hM, g.hR[:, None]),        # hR 2-D
        gen.ElsrInstance(g.D, g.R, g.kM, g.kR, g.hM, g.hR, g.kM[:2], None),  # pM too short
    ]
    for b in bad:
        with pytest.raises(ValueError):
            elsr.Solver(b)
        with pytest.raises(ValueError):
            elsr.Batch([g, b])


class _CaptureLib:
    """Stands in for the library: records what elsr_create / elsr_create_ex
    receive, reading the arrays behind the pointers during the call."""

    def __init__(self):
        self.calls = []

    def _read(self, ptr, n):
        buf = (ctypes.c_int32 * n).from_address(ptr.value if hasattr(ptr, "value") else ptr)
        return np.frombuffer(buf, dtype=np.int32).copy()

    def _create(self, name, out, K, T, *ptrs):
        arrays = [self._read(ptrs[0], K * T).reshape(K, T), self._read(ptrs[1], K * T).reshape(K, T)]
        arrays += [self._read(p, K) for p in ptrs[2:]]
        self.calls.append((name, K, T, arrays))
        return 0

    def elsr_create(self, out, K, T, *ptrs):
        return self._create("elsr_create", out, K, T, *ptrs)

    def elsr_create_ex(self, out, K, T, *ptrs):
        return self._create("elsr_create_ex", out, K, T, *ptrs)

    def elsr_set_stream(self, h, s):
        return 0

    def elsr_destroy(self, h):
        pass


def test_binding_passes_the_instance_in_abi_order(monkeypatch):
    """Solver hands elsr_create K, T and D, R, kM, kR, hM, hR (and pM, pR to
    elsr_create_ex) in the order include/elsr.h declares, as int32 copies of
    the instance's values."""
    from paper_1704_05132_gb300 import elsr, gen
    cap = _CaptureLib()
    monkeypatch.setattr(elsr, "load", lambda: cap)
    g = gen.make_instance(2, 5, K=3, T=7)
    gp = gen.with_production_costs(g, 4)
    for inst, name in ((g, "elsr_create"), (gp, "elsr_create_ex")):
        s = elsr.Solver(inst)
        s._h = None   # nothing to destroy in the stand-in
        got_name, K, T, arrays = cap.calls[-1]
        assert (got_name, K, T) == (name, 3, 7)
        fields = ["D", "R", "kM", "kR", "hM", "hR"] + (["pM", "pR"] if inst.pM is not None else [])
        assert len(arrays) == len(fields)
        for f, a in zip(fields, arrays):
            np.testing.assert_array_equal(a, getattr(inst, f), err_msg=f)


class _CaptureBatchLib(_CaptureLib):
    def _batch(self, name, out, n, Ks_p, Ts_p, *rest):
        Ks, Ts = self._read(Ks_p, n), self._read(Ts_p, n)
        cells, rows = int((Ks.astype(np.int64) * Ts).sum()), int(Ks.sum())
        ptrs = rest[:-1]  # the last argument is the stream
        arrays = [self._read(ptrs[0], cells), self._read(ptrs[1], cells)]
        arrays += [self._read(p, rows) for p in ptrs[2:]]
        self.calls.append((name, n, Ks, Ts, arrays))
        return 0

    def elsr_batch_create_on(self, out, n, Ks, Ts, *rest):
        return self._batch("elsr_batch_create_on", out, n, Ks, Ts, *rest)

    def elsr_batch_create_ex(self, out, n, Ks, Ts, *rest):
        return self._batch("elsr_batch_create_ex", out, n, Ks, Ts, *rest)

    def elsr_batch_destroy(self, b):
        pass


def test_batch_passes_instances_back_to_back(monkeypatch):
    """Batch hands the library n, Ks, Ts and the instances' arrays one after
    another ([K_i][T_i] cell blocks, [K_i] row blocks), zeros for the
    production costs of instances that have none."""
    from paper_1704_05132_gb300 import elsr, gen
    cap = _CaptureBatchLib()
    monkeypatch.setattr(elsr, "load", lambda: cap)
    insts = [gen.make_instance(3, i, K=k, T=t) for i, (k, t) in enumerate([(2, 5), (4, 3), (1, 9)])]
    mixed = [insts[0], gen.with_production_costs(insts[1], 6), insts[2]]
    for batch, name in ((insts, "elsr_batch_create_on"), (mixed, "elsr_batch_create_ex")):
        b = elsr.Batch(batch)
        b._b = None
        got, n, Ks, Ts, arrays = cap.calls[-1]
        assert (got, n) == (name, 3)
        assert Ks.tolist() == [2, 4, 1] and Ts.tolist() == [5, 3, 9]
        cells = ["D", "R"]
        rows = ["kM", "kR", "hM", "hR"] + (["pM", "pR"] if name.endswith("_ex") else [])
        for f, a in zip(cells + rows, arrays):
            if f in cells:
                want = np.concatenate([getattr(i, f).ravel() for i in batch])
            else:
                want = np.concatenate([getattr(i, f) if getattr(i, f) is not None
                                       else np.zeros(i.K, np.int32) for i in batch])
            np.testing.assert_array_equal(a, want, err_msg=f)


def test_server_config_is_validated_before_any_device_call(lib):
    """Invalid server configurations are refused with ELSR_E_ARG on the host
    (no device is touched), and the binding's structure has the header's
    size."""
    assert ctypes.sizeof(nat.ServerConfig) == 40
    h = ctypes.c_void_p()
    for field, value in (("slots", -1), ("threads", 100), ("threads", 2048), ("max_runs", -1),
                         ("acc64", 2), ("count_steps", -1), ("keep_solutions", 2)):
        cfg = nat.ServerConfig()
        setattr(cfg, field, value)
        assert lib.elsr_server_create(ctypes.byref(h), ctypes.byref(cfg)) == nat.ELSR_E_ARG, field
        assert not h.value
