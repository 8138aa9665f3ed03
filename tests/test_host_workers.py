"""The host set-up's worker threads (run_tasks / parallel_for in
csrc/hlbm_internal.h): set-ups run from several host threads at once give the
tables of a set-up run alone, and a process forked after the workers started
runs its own set-up to the same tables instead of waiting on threads it does
not have.  Host-only (hlbm_inspect needs no GPU)."""
import multiprocessing as mp
import threading

import numpy as np
import pytest

from workloads import make_case

TABLES = ("col", "cc", "is_don", "is_w", "perm")


@pytest.fixture(scope="module")
def H():
    from paper_2006_10487_gb300 import build
    build.build()
    import paper_2006_10487_gb300 as H
    return H


def _tables(H, case):
    return {t: H.hlbm_inspect(case, t) for t in TABLES}


def test_concurrent_setups_match_one_alone(H):
    case = make_case("hlbm_small", aoa_deg=5.0)
    ref = _tables(H, case)
    out, errors = [None] * 4, []

    def work(k):
        try:
            out[k] = _tables(H, case)
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not errors and all(not t.is_alive() for t in threads)
    for got in out:
        for t in TABLES:
            assert np.array_equal(got[t], ref[t]), t


def _child(q):
    import paper_2006_10487_gb300 as H
    case = make_case("hlbm_small", aoa_deg=5.0)
    q.put({t: H.hlbm_inspect(case, t).tobytes() for t in TABLES})


def test_forked_process_runs_its_own_setup(H):
    case = make_case("hlbm_small", aoa_deg=5.0)
    ref = _tables(H, case)  # the parent's workers are running now
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_child, args=(q,))
    p.start()
    try:
        got = q.get(timeout=120)
    finally:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    assert p.exitcode == 0
    for t in TABLES:
        assert got[t] == ref[t].tobytes(), t
