"""Register, stack and spill budget of the binary64 tall-pass kernels, read
from ptxas's resource report (-Xptxas -v) of the library's own build flags.

The FP64 passes are bound by GB300's FP64 pipe, and their launch plans
assume a number of resident CTAs per SM: two 256-thread CTAs for the TRSM,
the Gram and the Gaussian sketch (one CTA's TMA wait or barrier is covered by
the other), six for the tall LU's trailing update.  That only holds while
each thread's registers fit 65,536 / (CTAs x 256), allocated in units of 8
per thread; a spill or a local array would also put local-memory traffic on
the path.  These checks run on the CPU (nvcc cross-compiles sm_103a), so a
change that breaks the budget fails here before any GPU time is spent.
"""
import concurrent.futures
import os
import re
import shutil
import subprocess
import tempfile

import pytest

from paper_2412_06551_gb300 import _build

REGS_PER_SM = 65536


def _resources(sources):
    """{demangled kernel name: dict(regs, stack, spill_st, spill_ld)} for the
    given translation units, compiled as the library build compiles them."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    cxxfilt = shutil.which("c++filt")
    tmp = tempfile.mkdtemp(prefix="rq_ptxas_")

    def run(src):
        cmd = ([nvcc] + _build.ARCH + _build.FLAGS + ["-Xptxas", "-v", "-c",
               os.path.join(_build.CSRC, src), "-o", os.path.join(tmp, src + ".o")])
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        return r.stderr

    with concurrent.futures.ThreadPoolExecutor(len(sources)) as ex:
        logs = list(ex.map(run, sources))
    shutil.rmtree(tmp, ignore_errors=True)
    out, name = {}, None
    for log in logs:
        for line in log.splitlines():
            mt = re.search(r"Compiling entry function '([^']+)'", line)
            if mt:
                name = mt.group(1)
                if cxxfilt:
                    name = subprocess.run([cxxfilt, name], capture_output=True,
                                          text=True).stdout.strip()
                out[name] = {}
                continue
            mt = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
            if mt and name:
                out[name].update(stack=int(mt.group(1)), spill_st=int(mt.group(2)),
                                 spill_ld=int(mt.group(3)))
            mt = re.search(r"Used (\d+) registers", line)
            if mt and name:
                out[name]["regs"] = int(mt.group(1))
    return out


def _max_regs(threads, ctas_per_sm):
    """Largest per-thread register count that keeps ctas_per_sm CTAs of
    `threads` threads resident (allocation in units of 8 registers)."""
    return (REGS_PER_SM // (threads * ctas_per_sm)) // 8 * 8


def _const(src, name):
    txt = open(os.path.join(_build.CSRC, src)).read()
    return int(re.search(r"constexpr int %s = (\d+);" % name, txt).group(1))


@pytest.fixture(scope="module")
def res():
    r = _resources(["tall.cu", "lu.cu"])
    assert r, "ptxas reported no entry functions"
    return r


def _pick(res, pattern):
    hits = {k: v for k, v in res.items() if re.search(pattern, k)}
    assert hits, "no kernel matches %r" % pattern
    return hits


def test_fp64_tall_pass_kernels_do_not_spill(res):
    for name, r in res.items():
        assert r["spill_st"] == 0 and r["spill_ld"] == 0, (name, r)


def test_trsm_gram_and_gaussian_sketch_keep_state_in_registers(res):
    # the FP64-pipe-bound passes: no local memory at all, and two CTAs per SM
    threads = _const("tall.cu", "kThreads")
    cap = _max_regs(threads, 2)
    for pat in (r"\bk_trsm<", r"\bk_gram<\d+, 5>", r"\bk_sketch_gauss<"):
        for name, r in _pick(res, pat).items():
            assert r["stack"] == 0, (name, r)
            assert r["regs"] <= cap, (name, r, cap)


def test_off_diagonal_gram_keeps_its_eight_tiles_in_registers(res):
    # n > 128: the off-diagonal block runs one CTA per SM with eight warp tiles
    for name, r in _pick(res, r"\bk_gram<32, 8>").items():
        assert r["stack"] == 0, (name, r)


def test_lu_kernels_fit_their_planned_occupancy(res):
    threads = _const("lu.cu", "kLuThreads")
    per_sm = _const("lu.cu", "kTrailCtasPerSm")
    for name, r in _pick(res, r"\bk_lu_trailing\(").items():
        assert r["regs"] <= _max_regs(threads, per_sm), (name, r, per_sm)
    for name, r in _pick(res, r"\bk_lu_col\(").items():
        assert r["regs"] <= _max_regs(threads, 2), (name, r)


def test_budget_helper_matches_known_occupancies():
    # 256 threads: 2 CTAs -> 128 registers, 6 CTAs -> 40 (42 is not a unit of 8),
    # 1 CTA -> 255 is capped by the architecture, not by this formula
    assert _max_regs(256, 2) == 128
    assert _max_regs(256, 6) == 40
    assert _max_regs(128, 4) == 128
