"""CPU tests of the C-ABI library: it loads, exports and binds every function
that include/ac.h declares, validates its inputs, and its host builder (stage 1
of Sec. III.A, flattened) agrees with the oracle. No GPU is used: dfas are
built with AC_BUILD_HOST_ONLY and their tables are walked in Python."""
import os
import random
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from tests.conftest import ROOT, load_golden

HEADER = os.path.join(ROOT, "include", "ac.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(ac_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ("ac_build", "ac_scan", "ac_scan_batch", "ac_serve_create", "ac_serve_submit", "ac_serve_wait"):
        assert name in fns


def test_library_exports_every_declared_function():
    lib = acg.lib()
    nm = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (ac_\w+)$", nm, flags=re.M))
    for name in header_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_binding_covers_every_declared_function():
    assert sorted(N.SIGNATURES) == header_functions()


def test_status_strings():
    lib = acg.lib()
    for code in range(0, -12, -1):
        assert lib.ac_status_str(code).decode() != "unknown status"
    assert lib.ac_status_str(-99).decode() == "unknown status"


def test_struct_sizes_match_the_header():
    import ctypes

    assert ctypes.sizeof(N.Match) == 16
    assert ctypes.sizeof(N.Text) == 24
    assert ctypes.sizeof(N.Result) == 48
    assert ctypes.sizeof(N.ScanOpts) == 48
    assert ctypes.sizeof(N.ScanStats) == 56
    assert ctypes.sizeof(N.Served) == 40  # ac_served: two pointers, two counts, a handle


# ------------------------------------------------------------ validation


@pytest.mark.parametrize(
    "pats,code",
    [
        ([b"ACGT", b""], N.AC_ERR_EMPTY_PATTERN),
        ([b"ACGN"], N.AC_ERR_ALPHABET),
        ([b"acgt"], N.AC_ERR_ALPHABET),
        ([], N.AC_ERR_INVALID_ARG),
    ],
)
def test_build_rejects(pats, code):
    with pytest.raises(acg.AcError) as e:
        acg.build(pats, host_only=True)
    assert e.value.status == code


def test_fold_case_accepts_lower_case():
    d = acg.build([b"acgT"], fold_case=True, host_only=True)
    assert d.n_states == 5


def test_host_only_dfa_cannot_scan():
    import ctypes

    d = acg.build([b"ACGT"], host_only=True)
    t = N.Text(None, 0, N.AC_TEXT_ASCII, 0)
    r = N.Result()
    st = acg.lib().ac_scan(d.h, ctypes.byref(t), ctypes.byref(r), None, None, None)
    assert st == N.AC_ERR_NO_DEVICE


# ------------------------------------------- builder vs the oracle (CPU)

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def walk_tables(t, text: bytes):
    """One lookup per base over the flattened table; emits (start, pid)."""
    delta, off, pid, plen = t["delta"], t["out_off"], t["out_pid"], t["pat_len"]
    s, out = 0, set()
    for i, ch in enumerate(text):
        e = int(delta[4 * s + CODE[ch]])
        s = e & 0x7FFFFFFF
        if e >> 31:
            for k in range(off[s], off[s + 1]):
                p = int(pid[k])
                out.add((i + 1 - int(plen[p]), p))
        else:
            assert off[s] == off[s + 1], "flag bit clear on a state with output"
    return out


def strings_by_state(t):
    """string(s) for each breadth-first state, from the depth-increasing tree edges."""
    delta, depth = t["delta"].reshape(-1, 4), t["depth"]
    S = len(depth)
    s_of = {0: b""}
    for s in range(S):  # breadth-first ids: parents come first
        for c in range(4):
            nx = int(delta[s, c]) & 0x7FFFFFFF
            if depth[nx] == depth[s] + 1 and nx not in s_of:
                s_of[nx] = s_of[s] + b"ACGT"[c : c + 1]
    assert len(s_of) == S
    return s_of


def rand_set(rng, k, lo, hi):
    return [bytes(rng.choice(b"ACGT") for _ in range(rng.randint(lo, hi))) for _ in range(k)]


def test_worked_example_dna_tables():
    g = load_golden("worked_example_dna.txt")
    kws = [w.encode() for w in g["keywords"][0]]
    t = acg.build(kws, host_only=True).tables()
    got = walk_tables(t, g["text"][0][0].encode())
    assert got == {(int(p), [w.decode() for w in kws].index(k)) for p, k in g["match"]}


@pytest.mark.parametrize("seed", range(40))
def test_flattened_walk_equals_oracle(seed):
    rng = random.Random(500 + seed)
    pats = rand_set(rng, rng.randint(1, 60), 1, 9)
    if seed % 4 == 0:
        pats += [pats[0], pats[-1][:2] or b"A"]  # duplicates and prefixes
    n = rng.choice([0, 1, 50, 700, 3000])
    if seed % 5 == 0:
        text = (b"AC" * n)[:n]
    else:
        text = bytes(rng.choice(b"ACGT") for _ in range(n))
    d = acg.build(pats, host_only=True)
    t = d.tables()
    pos, pid, counts = oracle.Machine(pats).scan(text)
    assert walk_tables(t, text) == set(zip(pos.tolist(), pid.tolist()))


@pytest.mark.parametrize("seed", range(10))
def test_builder_fail_output_depth_match_oracle(seed):
    rng = random.Random(900 + seed)
    pats = rand_set(rng, rng.randint(1, 40), 1, 7)
    t = acg.build(pats, host_only=True).tables()
    m = oracle.Machine(pats)
    strings = strings_by_state(t)
    # the oracle's state for each string (walk its goto from the root)
    def orc_state(w):
        s = 0
        for c in w:
            s = m.goto(s, c)
        return s
    by_orc = {orc_state(w): s for s, w in strings.items()}
    assert len(by_orc) == m.n_states == len(strings)
    for s, w in strings.items():
        o = orc_state(w)
        assert t["depth"][s] == m.depth(o) == len(w)
        assert by_orc[m.fail(o)] == t["fail"][s]
        assert sorted(t["out_pid"][t["out_off"][s] : t["out_off"][s + 1]].tolist()) == sorted(m.output(o))
    for p, w in enumerate(pats):
        assert strings[int(t["pat_state"][p])] == w
        assert t["pat_len"][p] == len(w)


def walk_pairs(t, text: bytes):
    """Two bases per lookup over delta2; a keyword ending at the first base of
    a pair is found through bit 30 and one delta lookup, as the kernel does."""
    d1, d2, off, pid, plen = t["delta"], t["delta2"], t["out_off"], t["out_pid"], t["pat_len"]
    s, out = 0, set()

    def emit(state, end):
        for k in range(off[state], off[state + 1]):
            p = int(pid[k])
            out.add((end + 1 - int(plen[p]), p))

    rows = len(d2) // 16
    for i in range(0, len(text) - 1, 2):
        x, y = CODE[text[i]], CODE[text[i + 1]]
        if s < rows:
            e = int(d2[16 * s + (x | (y << 2))])
        else:  # no two-base row for this (deep) state: two one-base lookups
            e1 = int(d1[4 * s + x])
            e2 = int(d1[4 * (e1 & 0x3FFFFFFF) + y])
            e = e2 | ((e1 >> 31) << 30)
        if e & (1 << 30):
            emit(int(d1[4 * s + x]) & 0x3FFFFFFF, i)
        s = e & 0x3FFFFFFF
        if e >> 31:
            emit(s, i + 1)
    if len(text) % 2:  # odd tail: one single-base step
        e = int(d1[4 * s + CODE[text[-1]]])
        s = e & 0x3FFFFFFF
        if e >> 31:
            emit(s, len(text) - 1)
    return out


@pytest.mark.parametrize("seed", range(15))
@pytest.mark.parametrize("rows", [0, 1, 7])
def test_two_base_table_walk_equals_oracle(seed, rows):
    rng = random.Random(700 + seed)
    pats = rand_set(rng, rng.randint(1, 50), 1, 9)
    n = rng.choice([0, 1, 2, 3, 51, 700, 2001])
    text = bytes(rng.choice(b"ACGT") for _ in range(n)) if seed % 3 else (b"ACG" * n)[:n]
    t = acg.build(pats, host_only=True, stride2_states=rows).tables()
    assert len(t["delta2"]) == 16 * (min(rows, len(t["depth"])) if rows else len(t["depth"]))
    pos, pid, _ = oracle.Machine(pats).scan(text)
    assert walk_pairs(t, text) == set(zip(pos.tolist(), pid.tolist()))


def test_two_base_table_can_be_skipped():
    d = acg.build([b"ACGT"], host_only=True, stride2=False)
    assert d.info["table2_bytes"] == 0 and len(d.tables()["delta2"]) == 0


def walk_triples(t, text: bytes):
    """The three-base walk as the kernel takes it: from a state with a
    three-base row read three bases, from one with a two-base row two, else
    one; a keyword ending at the first or second base of a lookup is found
    through bit 29 / 30 (three-base rows) or bit 30 (two-base rows) and one or
    two delta lookups; bases past the text read as A and ends past it are
    dropped."""
    d1, d2, d3 = t["delta"], t["delta2"], t["delta3"]
    off, pid, plen = t["out_off"], t["out_pid"], t["pat_len"]
    rows2, rows3 = len(d2) // 16, len(d3) // 64
    M = 0x3FFFFFFF
    n = len(text)
    out = set()

    def emit(state, end):
        if end < n:
            for k in range(off[state], off[state + 1]):
                p = int(pid[k])
                out.add((end + 1 - int(plen[p]), p))

    codes = [CODE[c] for c in text] + [0, 0]
    s, i = 0, 0
    while i < n:
        x, y, z = codes[i], codes[i + 1], codes[i + 2]
        first = int(d1[4 * s + x]) & M
        if s < rows3:
            e = int(d3[64 * s + (x | (y << 2) | (z << 4))])
            if e & (1 << 29):
                emit(first, i)
            if e & (1 << 30):
                emit(int(d1[4 * first + y]) & M, i + 1)
            s, k = e & 0x1FFFFFFF, 3
        elif s < rows2:
            e = int(d2[16 * s + (x | (y << 2))])
            if e & (1 << 30):
                emit(first, i)
            s, k = e & M, 2
        else:
            e = int(d1[4 * s + x])
            s, k = e & M, 1
        if e >> 31:
            emit(s, i + k - 1)
        i += k
    return out


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("rows3", [None, 1, 7, 0])
@pytest.mark.parametrize("rows2", [0, 3])
def test_three_base_table_walk_equals_oracle(seed, rows3, rows2):
    rng = random.Random(750 + seed)
    pats = rand_set(rng, rng.randint(1, 50), 1, 9) + ([b"A", b"AA"] if seed % 2 else [])
    n = rng.choice([0, 1, 2, 3, 4, 5, 52, 701, 2000])
    text = bytes(rng.choice(b"ACGT") for _ in range(n)) if seed % 3 else (b"ACG" * n)[:n]
    d = acg.build(pats, host_only=True, stride2_states=rows2, stride3=rows3 is not None, stride3_states=rows3 or 0)
    t = d.tables()
    S = len(t["depth"])
    want3 = 0 if rows3 is None else (S if rows3 == 0 else min(rows3, S))
    assert len(t["delta3"]) == 64 * want3 and d.info["table3_bytes"] == 256 * want3
    pos, pid, _ = oracle.Machine(pats).scan(text)
    assert walk_triples(t, text) == set(zip(pos.tolist(), pid.tolist()))


def test_three_base_entries_compose_three_single_steps():
    rng = random.Random(77)
    t = acg.build(rand_set(rng, 30, 2, 8), host_only=True).tables()
    d1, d3 = t["delta"].astype(np.int64), t["delta3"].astype(np.int64)
    off = t["out_off"]
    has = lambda u: off[u + 1] > off[u]
    M = 0x3FFFFFFF
    for s in range(len(d3) // 64):
        for sym in range(64):
            x, y, z = sym & 3, (sym >> 2) & 3, sym >> 4
            a = int(d1[4 * s + x]) & M
            b = int(d1[4 * a + y]) & M
            c = int(d1[4 * b + z]) & M
            e = int(d3[64 * s + sym])
            assert e & 0x1FFFFFFF == c
            assert (e >> 31, (e >> 30) & 1, (e >> 29) & 1) == (int(has(c)), int(has(b)), int(has(a)))


def walk_failureless(t, text: bytes):
    """From every start, follow trie edges only and report own keywords."""
    g, off, pid = t["gotos"], t["own_off"], t["own_pid"]
    out = set()
    for i in range(len(text)):
        s = 0
        for j in range(i, len(text)):
            e = int(g[4 * s + CODE[text[j]]])
            if (e & 0x7FFFFFFF) == 0x7FFFFFFF:
                break
            s = e & 0x7FFFFFFF
            assert bool(e >> 31) == (off[s + 1] > off[s])
            out |= {(i, int(p)) for p in pid[off[s] : off[s + 1]]}
    return out


@pytest.mark.parametrize("seed", range(10))
def test_failureless_tables_walk_equals_oracle(seed):
    rng = random.Random(800 + seed)
    pats = rand_set(rng, rng.randint(1, 40), 1, 8) + [b"AAA", b"A"]
    text = bytes(rng.choice(b"ACGT") for _ in range(rng.choice([0, 1, 300, 1500]))) + b"AAAA"
    t = acg.build(pats, host_only=True, failureless=True).tables()
    pos, pid, _ = oracle.Machine(pats).scan(text)
    assert walk_failureless(t, text) == set(zip(pos.tolist(), pid.tolist()))
    assert "gotos" not in acg.build(pats, host_only=True).tables()


def test_breadth_first_numbering():
    rng = random.Random(3)
    t = acg.build(rand_set(rng, 200, 5, 12), host_only=True).tables()
    assert np.all(np.diff(t["depth"].astype(np.int64)) >= 0)  # depth non-decreasing in id order


def test_taken_result_views_release_once_when_the_last_view_dies(monkeypatch):
    """Server.wait without a capacity returns numpy views of the server's own copy
    (ac_serve_take); the copy is given back (ac_serve_release) exactly once, when neither
    the occurrence view nor the count view is referenced any more."""
    import ctypes
    import gc

    import numpy as np

    released = []

    class FakeLib:
        def ac_serve_release(self, h):
            released.append(h)

    monkeypatch.setattr(acg, "lib", lambda: FakeLib())
    occ = (ctypes.c_int64 * 6)(10, 1, 20, 2, 30, 3)
    cnt = (ctypes.c_int64 * 4)(0, 1, 1, 1)
    held = acg._Taken(12345)
    m = acg._view(ctypes.addressof(occ), 6, held).reshape(3, 2)
    c = acg._view(ctypes.addressof(cnt), 4, held)
    del held
    gc.collect()
    assert m.tolist() == [[10, 1], [20, 2], [30, 3]] and c.tolist() == [0, 1, 1, 1]
    assert released == []
    del m
    gc.collect()
    assert released == [] and c.sum() == 3
    del c
    gc.collect()
    assert released == [12345]
    assert acg._view(0, 0, None).shape == (0,)


def test_build_entry_leaves_the_public_build_function():
    """The in-tree compile step lives in a module whose import cannot shadow acg.build:
    building and then building a machine works in one process."""
    import __graft_entry__

    __graft_entry__.build()  # nothing to do when the library is current
    assert callable(acg.build)
    d = acg.build([b"ACGT", b"CG"], host_only=True)
    assert d.info["n_states"] == 7  # root, A, AC, ACG, ACGT, C, CG


def test_fault_plan_parsing_on_the_host():
    """ac_fault_inject needs no GPU: it only sets the host-side plan (cleared again here)."""
    lib = acg.lib()
    for spec in (b"oom@1", b"cuda_err@7", b"oom@3,cuda_err@2", b""):
        assert lib.ac_fault_inject(spec) == N.AC_OK
    for bad in (b"oom", b"oom@0", b"oom@-2", b"oom@x", b"leak@1", b"oom@1;cuda_err@2", b"oom@1,"):
        assert lib.ac_fault_inject(bad) == N.AC_ERR_INVALID_ARG
    assert lib.ac_fault_inject(None) == N.AC_OK


# C type of each ctypes mirror in _native.py
C_STRUCTS = {"BuildOpts": "ac_build_opts", "DfaInfo": "ac_dfa_info_t", "DfaTables": "ac_dfa_tables_t", "Text": "ac_text",
             "Match": "ac_match", "Result": "ac_result", "ScanOpts": "ac_scan_opts", "ScanStats": "ac_scan_stats",
             "ServeOpts": "ac_serve_opts", "Served": "ac_served", "ServeStats": "ac_serve_stats_t",
             "MemUsage": "ac_mem_usage_t"}


def test_binding_structs_match_the_c_header(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C compiler gives the
    header's struct (compiled here with gcc)."""
    import ctypes
    import shutil

    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for py, c in C_STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(N, py)._fields_:
            lines.append(f'printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            py, name, v = line.split()
            got[(py, name)] = int(v)
    for py in C_STRUCTS:
        cls = getattr(N, py)
        assert got[(py, "size")] == ctypes.sizeof(cls), py
        for name, _ in cls._fields_:
            assert got[(py, name)] == getattr(cls, name).offset, (py, name)


def test_library_carries_its_nvtx_ranges():
    """The entry points open NVTX ranges in the acgpu domain (names compiled into libac.so)."""
    blob = open(N.LIB_PATH, "rb").read()
    for name in (b"acgpu", b"ac_scan", b"ac_scan_batch", b"ac_batch_plan_run", b"ac_stream_scan",
                 b"ac_serve batch", b"ac_autotune"):
        assert name + b"\x00" in blob, name
