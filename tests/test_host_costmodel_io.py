"""Host-only checks (no GPU) of the cost-model file entry points and of the
allocation-failure test hook.

- qsa_costmodel_save / qsa_costmodel_load round-trip a network exactly (the
  parameters are FP32 in the file and in the library), a NULL path removes
  the process-wide model, and malformed files (wrong header, wrong count,
  truncated, trailing bytes, a non-finite parameter) are refused without
  changing the installed model.
- qsa_debug_fail_alloc makes the next device allocation fail on the host:
  state creation returns QSA_E_NOMEM with the out-of-memory message, holds
  nothing afterwards, and the hook is spent after one failure; the
  QSA_FAULT_ALLOC environment variable does the same at load time.
"""
import os
import struct
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def q():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2608_16940_gb300 as q
    return q


def _features(q, rng, count=40):
    X = np.zeros((count, 37), dtype=np.float32)
    for i in range(count):
        k = int(rng.integers(1, 7))
        mask = 0
        for t in rng.choice(30, size=k, replace=False):
            mask |= 1 << int(t)
        X[i] = q.qsa_costmodel_features(k, mask, 30, 1)
    return X


def test_model_file_round_trip(q, tmp_path):
    rng = np.random.default_rng(1)
    params = q.qsa_costmodel_init(5) * np.float32(0.3)
    X = _features(q, rng)
    q.qsa_costmodel_set(params)
    try:
        want = q.qsa_costmodel_predict(X)
        path = str(tmp_path / "model.qsacm")
        q.qsa_costmodel_save(path)
        raw = open(path, "rb").read()
        assert raw[:8] == b"QSACM001" and struct.unpack("<I", raw[8:12])[0] == q.MLP_PARAMS
        assert np.array_equal(np.frombuffer(raw[12:], dtype="<f4"), params)
        q.qsa_costmodel_load(None, None)          # remove
        with pytest.raises(q.QsaError) as e:
            q.qsa_costmodel_predict(X)
        assert e.value.code == q.QSA_E_STATE
        q.qsa_costmodel_load(None, path)          # install from the file
        assert np.array_equal(q.qsa_costmodel_predict(X), want)
    finally:
        q.qsa_costmodel_set(None)


def test_save_without_model_is_a_state_error(q, tmp_path):
    q.qsa_costmodel_set(None)
    with pytest.raises(q.QsaError) as e:
        q.qsa_costmodel_save(str(tmp_path / "none.qsacm"))
    assert e.value.code == q.QSA_E_STATE


@pytest.mark.parametrize("case", ["magic", "count", "truncated", "trailing", "nan", "missing"])
def test_malformed_model_files_are_refused(q, tmp_path, case):
    good = np.linspace(-1, 1, q.MLP_PARAMS).astype("<f4")
    head, cnt, body = b"QSACM001", struct.pack("<I", q.MLP_PARAMS), good.tobytes()
    if case == "magic":
        head = b"QSACM002"
    elif case == "count":
        cnt = struct.pack("<I", q.MLP_PARAMS - 1)
    elif case == "truncated":
        body = body[:-4]
    elif case == "trailing":
        body = body + b"\0"
    elif case == "nan":
        bad = good.copy()
        bad[17] = np.nan
        body = bad.tobytes()
    path = str(tmp_path / f"{case}.qsacm")
    if case != "missing":
        open(path, "wb").write(head + cnt + body)
    params = q.qsa_costmodel_init(3)
    q.qsa_costmodel_set(params)
    try:
        X = _features(q, np.random.default_rng(2), 5)
        before = q.qsa_costmodel_predict(X)
        with pytest.raises(q.QsaError) as e:
            q.qsa_costmodel_load(None, path)
        assert e.value.code == q.QSA_E_ARG
        assert np.array_equal(q.qsa_costmodel_predict(X), before)   # nothing changed
    finally:
        q.qsa_costmodel_set(None)


def test_injected_allocation_failure_returns_nomem_and_holds_nothing(q):
    live = q.qsa_debug_live_allocations()
    q.qsa_debug_fail_alloc(0)
    try:
        with pytest.raises(q.QsaError) as e:
            q.qsa_state_create(10)
        assert e.value.code == q.QSA_E_NOMEM and "out of memory" in str(e.value)
        assert q.qsa_debug_live_allocations() == live
    finally:
        q.qsa_debug_fail_alloc(-1)


def test_fault_environment_variable(q):
    """QSA_FAULT_ALLOC=0 in a fresh process: its first state creation fails
    with QSA_E_NOMEM before any device call is made."""
    code = ("import paper_2608_16940_gb300 as q\n"
            "try:\n    q.qsa_state_create(8)\nexcept q.QsaError as e:\n"
            "    print('code', e.code, 'live', q.qsa_debug_live_allocations())\n")
    env = dict(os.environ, QSA_FAULT_ALLOC="0")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert f"code {q.QSA_E_NOMEM} live 0" in out.stdout, out.stdout
