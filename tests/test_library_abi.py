"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/rclupp.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

import paper_2412_06551_gb300 as rq
from paper_2412_06551_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = set()
    for h in hdrs:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for mt in re.finditer(r"\b(?:rclupp_status_t|const char \*|void|int|unsigned long long)\s*\*?\s*(\w+)\s*\(", txt):
            names.add(mt.group(1))
    return names


def test_library_builds_and_loads():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    assert lib is not None


def test_every_declared_symbol_is_exported():
    declared = _declared()
    assert {"rclupp_factor", "rclupp_r_factor", "cholqr2_factor", "lc2_factor"} <= declared
    lib = ctypes.CDLL(_build.build())
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(rq.exported_symbols()) == _declared()


def test_status_strings_without_gpu():
    lib = rq.load()
    assert lib.rclupp_status_string(0) == b"ok"
    assert lib.rclupp_status_string(-2) == b"Cholesky breakdown"


def test_argument_errors_before_any_gpu_work():
    # NULL handle / bad sizes are rejected on the host, with no CUDA call.
    lib = rq.load()
    info = rq.Info()
    st = lib.cholqr2_factor(None, 10, 4, None, 10, None, 10, None, 4, ctypes.byref(info))
    assert st == rq.Status.ERR_ARG
    assert lib.rclupp_create(None, None) == rq.Status.ERR_ARG


def test_no_cpu_fallback_in_the_binding():
    torch = pytest.importorskip("torch")
    x = torch.zeros((8, 2), dtype=torch.float64)
    with pytest.raises(TypeError):
        rq.cholqr2_factor(x)


def test_workspace_size_query_needs_no_gpu():
    # a host-only query: grows with the sketch size and adds the m x n LU copy
    # exactly when RCLUPPr / LC2 cannot factor in the Q buffer
    m, n = 100000, 64
    a = rq.workspace_size(rq.ALGO_RCLUPP, m, n)
    b = rq.workspace_size(rq.ALGO_RCLUPP, m, n, s=4 * n)
    assert 0 < a <= b
    lu = rq.workspace_size(rq.ALGO_RCLUPPR, m, n)
    lu_alias = rq.workspace_size(rq.ALGO_RCLUPPR, m, n, q_aliases_x=True)
    assert lu_alias - lu >= m * n * 8
    assert rq.workspace_size(rq.ALGO_LC2, m, n, q_aliases_x=True) - rq.workspace_size(rq.ALGO_LC2, m, n) >= m * n * 8
    assert rq.workspace_size(rq.ALGO_RCLUPPR, m, n, prec=rq.PREC_EMULATED) >= lu_alias - 256
    # sized for the GB300's 152 SMs: per-CTA partial sums of up to 2 * 152 + 8
    # CTAs (three 128 x 128 Gram slots; an s x n sketch tile at s = 4096)
    slots = 2 * 152 + 8
    assert a >= slots * 3 * 128 * 128 * 8
    assert rq.workspace_size(rq.ALGO_RCLUPP, 10 ** 6, 256, s=4096) >= slots * 4096 * 256 * 8
    with pytest.raises(rq.RclupError):
        rq.workspace_size(rq.ALGO_RCLUPP, 10, 20)        # m < n
    with pytest.raises(rq.RclupError):
        rq.workspace_size(rq.ALGO_RCLUPP, 1000, 300)     # n > 256


def test_product_sources_never_reach_the_oracle():
    # the package and its CUDA sources name neither the oracle nor the input
    # generators: no import, no include, no path
    import ast
    pkg = os.path.join(ROOT, "paper_2412_06551_gb300")
    checked = 0
    for dirpath, dirs, files in os.walk(pkg):
        dirs[:] = [d for d in dirs if d not in ("_build", "__pycache__")]
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        names = [a.name for a in node.names]
                    elif isinstance(node, ast.ImportFrom):
                        names = [node.module or ""]
                    else:
                        continue
                    assert not any(nm.split(".")[0] in ("oracle", "synth") for nm in names), (path, names)
            elif f.endswith((".cu", ".cuh", ".h", ".c", ".cpp")):
                src = open(path).read().lower()
                assert "oracle" not in src and "synth" not in src, path
            else:
                continue
            checked += 1
    assert checked >= 15


def test_missing_library_fails_loudly(tmp_path):
    import subprocess
    import sys
    code = ("import paper_2412_06551_gb300 as rq\n"
            "from paper_2412_06551_gb300 import _build\n"
            "_build.LIB = %r\n"
            "try:\n"
            "    rq.load(build=False)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n") % str(tmp_path / "absent.so")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "raised: librclupp.so is missing" in r.stdout


_ARG_SCRIPT = r'''
import ctypes, json, sys
import paper_2412_06551_gb300 as rq
lib = rq.load()
# argument checks run before the handle or any pointer is used: a zeroed
# host block stands in for the handle and the matrices
block = ctypes.create_string_buffer(1 << 16)
h = ctypes.c_void_p(ctypes.addressof(block))
X = Q = R = ctypes.c_void_p(ctypes.addressof(block))
info = rq.Info()
def opts(**kw):
    o = rq.Opts()
    o.kind, o.zeta, o.s, o.seed, o.prec = 0, 8, 0, 0, 0
    for k, v in kw.items():
        setattr(o, k, v)
    return o
out = {}
rand = {"rclupp": lib.rclupp_factor, "rcluppr": lib.rclupp_r_factor, "rcholqr": lib.rcholqr_factor}
plain = {"cholqr2": lib.cholqr2_factor, "lc2": lib.lc2_factor, "scholqr3": lib.scholqr3_factor}
sizes = {"n0": (10, 0, 10, 10, 1), "m0": (0, 1, 1, 1, 1), "m_lt_n": (3, 5, 3, 3, 5),
         "ldx_lt_m": (10, 4, 9, 10, 4), "ldq_lt_m": (10, 4, 10, 9, 4), "ldr_lt_n": (10, 4, 10, 10, 3),
         "n_257": (600, 257, 600, 600, 257), "m_2_31": (1 << 31, 4, 1 << 31, 1 << 31, 4)}
for name, f in list(rand.items()) + list(plain.items()):
    for case, (m, n, ldx, ldq, ldr) in sizes.items():
        args = (h, m, n, X, ldx) + ((None,) if name in rand else ()) + (Q, ldq, R, ldr, ctypes.byref(info))
        out[name + ":" + case] = f(*args)
for name, f in rand.items():
    for case, o in {"s_lt_n": opts(s=3), "s_4097": opts(s=4097), "kind_7": opts(s=8, kind=7),
                    "prec_9": opts(s=8, prec=9), "r0_5": opts(s=8, r0_method=5),
                    "zeta_0": opts(s=8, kind=1, zeta=0), "zeta_17": opts(s=64, kind=1, zeta=17),
                    "sparse_s_769": opts(s=769, kind=1, zeta=8), "srht_b_40": opts(s=8, kind=2, order_log2=40),
                    "srht_order_too_small": opts(s=8, kind=2, order_log2=3),
                    "explicit_lds_lt_s": opts(s=8, S=ctypes.addressof(block), lds=7),
                    "givens_too_big": opts(s=4096, r0_method=1)}.items():
        out[name + ":" + case] = f(h, 10000, 4 if case != "givens_too_big" else 256, X, 10000,
                                   ctypes.byref(o), Q, 10000, R, 256, ctypes.byref(info))
print(json.dumps(out))
'''


def test_argument_errors_are_found_before_the_handle_is_used():
    # every driver rejects bad sizes, leading dimensions and options on the
    # host, before it touches the handle, the matrices or the GPU (run in a
    # subprocess: a check that let a case through would reach the dummy handle)
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _ARG_SCRIPT], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    ARG, UNSUP = rq.Status.ERR_ARG, rq.Status.ERR_UNSUPPORTED
    expect_unsup = ("n_257", "m_2_31", "s_4097", "zeta_17", "sparse_s_769", "givens_too_big")
    assert len(out) == 6 * 8 + 3 * 12
    for key, st in out.items():
        case = key.split(":")[1]
        assert st == (UNSUP if case in expect_unsup else ARG), (key, st)


def test_each_thread_gets_its_own_handle_per_device(monkeypatch):
    """A handle serves one call at a time (one stream binding, one workspace),
    and the C calls run without the GIL, so the binding keeps one handle per
    (host thread, device).  A stand-in Handle records what was created."""
    import threading

    import torch

    made = []

    class FakeHandle:
        def __init__(self, device):
            self.device = torch.device(device)
            made.append(self)

    monkeypatch.setattr(rq, "Handle", FakeHandle)
    monkeypatch.setattr(rq, "_local", threading.local())

    class FakeTensor:
        def __init__(self, dev):
            self.device = torch.device(dev)

    h0 = rq._device_handle("cuda:0")
    assert rq._device_handle("cuda:0") is h0
    assert rq._handle(FakeTensor("cuda:0")) is h0
    h1 = rq._device_handle("cuda:1")
    assert h1 is not h0 and h1.device == torch.device("cuda:1")

    other = {}

    def worker():
        other["h0"] = rq._device_handle("cuda:0")
        other["again"] = rq._handle(FakeTensor("cuda:0"))

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert other["h0"] is other["again"]
    assert other["h0"] is not h0 and other["h0"].device == torch.device("cuda:0")
    assert len(made) == 3
    # the main thread's handles are unchanged by the other thread
    assert rq._device_handle("cuda:0") is h0


def test_every_entry_point_cites_its_passage_or_says_it_has_none():
    """Each declaration in include/*.h is preceded by a comment (or sits under
    a section banner) that names the passage of the paper defining the
    operation, or states that the paper has no counterpart."""
    cite = re.compile(r"Section \d|Algorithms? \d|eq\. \(|Lemma \d|Theorem \d|\bC\d\b|"
                      r"no counterpart in the paper")
    decl = re.compile(r"^(?:rclupp_status_t|const char \*|void|int|unsigned long long)\s*\*?\s*"
                      r"(\w+)\s*\(", re.M)
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fname)).read()
        comments = [(mt.start(), mt.end(), mt.group(0)) for mt in re.finditer(r"/\*.*?\*/", txt, re.S)]
        banners = [c for c in comments if c[2].startswith("/* ----")]
        for mt in decl.finditer(txt):
            before = [c for c in comments if c[1] <= mt.start()]
            assert before, mt.group(1)
            own = before[-1][2]
            banner = [b[2] for b in banners if b[1] <= mt.start()]
            ok = cite.search(own) or (banner and cite.search(banner[-1]))
            assert ok, "%s: %s has no citation" % (fname, mt.group(1))


def test_batched_arguments_keep_every_pointer_target_alive(monkeypatch):
    """The batched binding passes device pointers of column-major copies when
    an input comes in another layout; those copies must stay referenced until
    the C call returns, not go back to the allocator when the argument
    builder returns.  Stand-ins replace the layout copy and the handle."""
    import torch

    made = []

    def fake_colmajor(t):
        c = t.clone()  # stands in for the layout copy
        made.append(c)
        return c, t.shape[0]

    class FakeHandle:
        def bind(self):
            return None

    monkeypatch.setattr(rq, "colmajor", fake_colmajor)
    monkeypatch.setattr(rq, "_handle", lambda t: FakeHandle())
    shapes = [(5, 2), (7, 3)]
    Xs = [torch.zeros(s, dtype=torch.float64) for s in shapes]
    Qs = [torch.zeros(s, dtype=torch.float64) for s in shapes]
    Rs = [torch.zeros((s[1], s[1]), dtype=torch.float64) for s in shapes]
    a = rq._batch_args(Xs, Qs, Rs, None, rq.SKETCH_GAUSSIAN, 8, 0)
    del Xs, Qs, Rs

    def refs(obj, out):
        if isinstance(obj, (list, tuple)):
            for o in obj:
                refs(o, out)
        else:
            out.append(obj)
        return out

    held = refs([a["keep"], a["Qs"], a["Rs"]], [])
    passed = {int(p) for arr in (a["keep"][2], a["keep"][5], a["keep"][7]) for p in arr}
    assert len(made) == 6
    for c in made:
        assert c.data_ptr() in passed
        assert any(c is h for h in held), "a tensor whose pointer is passed is not kept"


def test_profiler_classes_agree_across_header_library_and_binding():
    """The kernel classes rclupp_profile_get names (callable without a GPU
    while nothing is pending), the list in include/rclupp.h and the
    binding's KERNEL_CLASSES are the same, in the same order."""
    lib = ctypes.CDLL(_build.build())
    lib.rclupp_profile_get.restype = ctypes.c_int
    lib.rclupp_profile_get.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_char_p)]
    names = []
    for k in range(64):
        nm = ctypes.c_char_p()
        st = lib.rclupp_profile_get(k, None, None, ctypes.byref(nm))
        if st != 0:
            assert st == rq.Status.ERR_ARG
            break
        names.append(nm.value.decode())
    assert names == rq.KERNEL_CLASSES
    txt = open(os.path.join(ROOT, "include", "rclupp.h")).read()
    block = txt[txt.index("rclupp_profile_get synchronizes"):txt.index("void rclupp_profile_enable")]
    block = re.sub(r"\s*\*\s*", " ", block)
    assert "0 <= kid < %d" % len(names) in block
    listed = re.findall(r"\b(\d+) ([a-z_0-9]+)", block[block.index("Classes:"):])
    assert [(int(i), nm) for i, nm in listed] == list(enumerate(names))
