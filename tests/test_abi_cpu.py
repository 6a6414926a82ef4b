"""Host-side checks of the C ABI: the library loads, exports every function
include/spcg.h declares, and its host-only entry points (no CUDA call)
agree with the oracle's schedule reading of Sec. 4."""
import ctypes
import os

import pytest

from oracle.spcg import default_schedule
from paper_2607_25272_b300 import spcg as S


def test_library_exports_every_declared_symbol():
    L = S.lib()
    names = S.declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(S._SIGS)


def test_status_strings():
    for code, name in S.STATUS.items():
        assert S.status_str(code) == name
    assert S.status_str(99) == "SPCG_E_UNKNOWN"


@pytest.mark.parametrize("N,d", [(20000, 50), (1 << 20, 500), (1 << 22, 1000), (1 << 23, 256),
                                 (3000, 37), (100, 50), (5000, 1), (1 << 17, 64)])
def test_default_schedule_matches_oracle_reading(N, d):
    s = S.spcg_default_schedule(N, d)
    o = default_schedule(N, d)
    assert list(s.m[: s.K]) == o["m"]
    assert list(s.a[: s.K]) == o["a"]
    assert s.r == min(o["r"], o["n_pad"])
    assert s.tol == 1e-6 and s.max_iters == 100


@pytest.mark.parametrize("N,d", [(1 << 22, 64), (1 << 20, 500), (20000, 50), (1 << 23, 256)])
def test_tuned_schedule_matches_oracle_reading(N, d):
    from oracle.spcg import tuned_schedule
    s = S.spcg_tuned_schedule(N, d)
    o = tuned_schedule(N, d)
    assert list(s.m[: s.K]) == o["m"] and list(s.a[: s.K]) == o["a"] and s.r == o["r"]


def test_invalid_arguments_rejected_before_any_cuda_call():
    L = S.lib()
    out = ctypes.c_void_p()
    # null X / Y, d out of range, N <= d: SPCG_E_INVALID_ARG, ctx stays NULL
    assert L.spcg_create(None, None, 100, 5, 5, None, None, ctypes.byref(out)) == S.SPCG_E_INVALID_ARG
    assert out.value is None
    fake = ctypes.c_void_p(16)
    assert L.spcg_create(fake, fake, 100, 0, 5, None, None, ctypes.byref(out)) == S.SPCG_E_INVALID_ARG
    assert L.spcg_create(fake, fake, 5, 5, 5, None, None, ctypes.byref(out)) == S.SPCG_E_INVALID_ARG
    assert L.spcg_create(fake, fake, 100, 2000, 2000, None, None, ctypes.byref(out)) == S.SPCG_E_INVALID_ARG
    assert L.spcg_create(fake, fake, 100, 5, 4, None, None, ctypes.byref(out)) == S.SPCG_E_INVALID_ARG
    sch = S.Schedule()
    assert L.spcg_default_schedule(10, 10, ctypes.byref(sch)) == S.SPCG_E_INVALID_ARG
    assert L.spcg_default_schedule(10, 3, None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_sketch(None, 1, None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_pcg_stage(None, 0, 1, None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_solve(None, 1, None, None, None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_feistel(1, 31, 0, 1, 0, None, None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_feistel(1, 4, 0, 17, 0, fake, None) == S.SPCG_E_INVALID_ARG
    # residual and split entry points: null context, bad operand type, odd strides,
    # misaligned pointers
    assert L.spcg_resid_apply_typed(None, fake, 0, 10, 10, fake, fake, fake) == S.SPCG_E_INVALID_ARG
    assert L.spcg_gram_apply_typed(None, fake, 4, 10, 10, fake, fake) == S.SPCG_E_INVALID_ARG
    f16 = ctypes.c_void_p(1 << 20)
    assert L.spcg_split_f32(f16, 10, 5, 5, f16, f16, 6, None) == S.SPCG_E_INVALID_ARG    # odd ldx
    assert L.spcg_split_f32(f16, 10, 5, 6, f16, f16, 5, None) == S.SPCG_E_INVALID_ARG    # odd ldxf
    assert L.spcg_split_f32(ctypes.c_void_p((1 << 20) + 8), 10, 5, 6, f16, f16, 6,
                            None) == S.SPCG_E_INVALID_ARG                              # X not 16-B
    assert L.spcg_split_f32(f16, 10, 5, 4, f16, f16, 6, None) == S.SPCG_E_INVALID_ARG    # ldx < d
    assert L.spcg_split_f32(f16, -1, 5, 6, f16, f16, 6, None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_split_f32(None, 0, 5, 6, None, None, 6, None) == S.SPCG_OK             # N = 0
    # the allocation-free pass checks its arguments before any CUDA call
    assert L.spcg_gram_apply_noalloc(f16, 10, 0, 10, f16, f16, None) == S.SPCG_E_INVALID_ARG   # d = 0
    assert L.spcg_gram_apply_noalloc(f16, 10, 1025, 1026, f16, f16,
                                     None) == S.SPCG_E_INVALID_ARG                          # d > 1024
    assert L.spcg_gram_apply_noalloc(f16, 10, 8, 7, f16, f16, None) == S.SPCG_E_INVALID_ARG    # lda < d
    assert L.spcg_gram_apply_noalloc(f16, 10, 8, 8, None, f16, None) == S.SPCG_E_INVALID_ARG   # p NULL
    assert L.spcg_gram_apply_noalloc(f16, 10, 8, 8, f16, None, None) == S.SPCG_E_INVALID_ARG   # w NULL
    assert L.spcg_gram_apply_noalloc(None, 10, 8, 8, f16, f16, None) == S.SPCG_E_INVALID_ARG   # A NULL
    assert L.spcg_gram_apply_noalloc(f16, -1, 8, 8, f16, f16, None) == S.SPCG_E_INVALID_ARG    # m < 0
    # the FMA probe: bad type, no iterations, NULL output
    out_d = ctypes.c_double(0.0)
    assert L.spcg_probe_fma_tflops(2, 10, ctypes.byref(out_d), None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_probe_fma_tflops(0, 0, ctypes.byref(out_d), None) == S.SPCG_E_INVALID_ARG
    assert L.spcg_probe_fma_tflops(0, 10, None, None) == S.SPCG_E_INVALID_ARG
    L.spcg_destroy(None)   # no-op


@pytest.mark.parametrize("field,value", [("precision", 2), ("precision", -1), ("fwht_tile", 4),
                                         ("fwht_tile", -1), ("fwht_first_levels", 13),
                                         ("fwht_first_levels", -1), ("max_workspace_bytes", -1),
                                         ("qr_panel_ctas", -1), ("dspace_ctas", -1),
                                         ("qr_by_column", 3), ("qr_by_column", -1)])
def test_options_out_of_range_rejected_before_any_cuda_call(field, value):
    """Every spcg_opts field outside its documented range gives
    SPCG_E_INVALID_ARG from spcg_create and spcg_solve_host before any CUDA
    call (so also on a host without a GPU); the context stays NULL."""
    L = S.lib()
    o = S.Opts()
    setattr(o, field, value)
    out = ctypes.c_void_p()
    fake = ctypes.c_void_p(16)
    assert L.spcg_create(fake, fake, 100, 5, 5, None, ctypes.byref(o),
                         ctypes.byref(out)) == S.SPCG_E_INVALID_ARG
    assert out.value is None
    sch = S.Schedule()
    assert L.spcg_default_schedule(100, 5, ctypes.byref(sch)) == S.SPCG_OK
    # X, Y, N, d, ldx, seed, sched, opts, stream, beta, info
    assert L.spcg_solve_host(fake, fake, 100, 5, 5, ctypes.c_uint64(1), ctypes.byref(sch),
                             ctypes.byref(o), None, fake, None) == S.SPCG_E_INVALID_ARG


def test_struct_layouts_match_header_sizes():
    # spcg_schedule: int32 K, int64 m[40], int32 a[40], int64 r, double tol, 2 x int32
    assert ctypes.sizeof(S.Schedule) == 8 + 8 * 40 + 4 * 40 + 8 + 8 + 8 + 8
    # spcg_opts: int32 precision, grid_ctas; int64 spin_budget; 4 x int32; int64 cap;
    # int32 qr_by_column, fwht_tile, fwht_first_levels, qr_panel_ctas, dspace_ctas
    # (+ 4 bytes of tail padding to the int64 alignment)
    assert ctypes.sizeof(S.Opts) == 4 + 4 + 8 + 16 + 8 + 20 + 4


def test_struct_layouts_match_a_c_compiler(tmp_path):
    """sizeof and field offsets as gcc lays out the structs of include/spcg.h."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"spcg_schedule": S.Schedule, "spcg_opts": S.Opts, "spcg_info": S.Info,
               "spcg_problem_f32": S.ProblemF32}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "spcg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


@pytest.mark.parametrize("N,d", [(1 << 20, 64), (70000, 129), (1 << 23, 256), (5000, 37)])
def test_candidate_schedules_enumerate_the_learned_choice_set(N, d):
    """The 25 candidates of the learned schedule: candidate 0 keeps only the
    paper's first stage; candidate 1 + 6(g-1) + 3(s-1) + (a-2) adds stages
    that grow by 2^s from the first up to N'/2^g, a iterations each
    (g = 1..4, s = 1, 2, a = 2, 3, 4); candidate 2 is the paper's schedule."""
    from oracle.spcg import default_schedule
    paper = default_schedule(N, d)
    n_pad = paper["n_pad"]
    seen = set()
    for idx in range(25):
        c = S.spcg_candidate_schedule(N, d, idx)
        m, a = list(c.m[: c.K]), list(c.a[: c.K])
        if not paper["m"]:
            assert c.K == 0
            continue
        m1 = paper["m"][0]
        assert m[0] == m1 and a[0] == 3
        if idx == 0:
            assert c.K == 1
        else:
            g, rem = 1 + (idx - 1) // 6, (idx - 1) % 6
            s, ai = 1 + rem // 3, 2 + rem % 3
            want, mm = [m1], m1 << s
            while mm <= n_pad >> g:
                want.append(mm)
                mm <<= s
            assert m == want and a == [3] + [ai] * (len(want) - 1)
        assert all(x <= n_pad // 2 for x in m)
        seen.add(tuple(m + a))
    if paper["m"]:
        c2 = S.spcg_candidate_schedule(N, d, 2)
        assert list(c2.m[: c2.K]) == paper["m"] and list(c2.a[: c2.K]) == paper["a"]
    with pytest.raises(S.SpcgError):
        S.spcg_candidate_schedule(N, d, 25)


def test_batched_and_model_entry_points_reject_bad_arguments():
    """The batched solver, the schedule model's kernels, the random maps and
    the context-level calls check their arguments before any CUDA call."""
    L = S.lib()
    E = S.SPCG_E_INVALID_ARG
    a16 = ctypes.c_void_p(1 << 20)            # a 16-byte-aligned stand-in address

    def prob(**kw):
        q = S.ProblemF32(X=a16, Y=a16, N=1000, d=16, ldx=16, beta=a16)
        for k, v in kw.items():
            setattr(q, k, v)
        return q

    out = ctypes.c_void_p()
    bad = [dict(d=0), dict(d=257, ldx=260), dict(N=16), dict(N=(1 << 24) + 1), dict(ldx=15),
           dict(ldx=18), dict(X=ctypes.c_void_p((1 << 20) + 4)), dict(X=None), dict(Y=None),
           dict(beta=None)]
    for kw in bad:
        arr = (S.ProblemF32 * 2)(prob(), prob(**kw))     # the bad one second
        assert L.spcg_batch_create(arr, 2, None, ctypes.byref(out)) == E, kw
        assert out.value is None
        st = (ctypes.c_int32 * 2)()
        assert L.spcg_solve_batched(arr, 2, 1, 1e-6, None, st, st) == E, kw
    arr = (S.ProblemF32 * 1)(prob())
    assert L.spcg_batch_create(arr, 0, None, ctypes.byref(out)) == E
    assert L.spcg_batch_create(None, 1, None, ctypes.byref(out)) == E
    assert L.spcg_batch_create(arr, 1, None, None) == E
    tiles = (ctypes.c_int32 * 4)()
    assert L.spcg_batch_solve(None, 1, 1e-6, None, None, None) == E
    assert L.spcg_batch_set_tiles(None, tiles) == E
    assert L.spcg_batch_autotune(None, 1, 1e-6, tiles) == E
    assert L.spcg_batch_phase_cycles(None, (ctypes.c_int64 * 8)()) == E
    L.spcg_batch_destroy(None)   # no-op
    # schedule model: sizes, output widths, NULL buffers
    assert L.spcg_num_candidates() == 25
    assert L.spcg_mlp_params(0) == -1 and L.spcg_mlp_params(1000) == -1
    assert L.spcg_mlp_params(25) > 0
    assert L.spcg_mlp_workspace_floats(25, -1) == -1 and L.spcg_mlp_workspace_floats(0, 4) == -1
    assert L.spcg_mlp_forward(None, 25, a16, 4, a16, None) == E
    assert L.spcg_mlp_forward(a16, 0, a16, 4, a16, None) == E
    assert L.spcg_mlp_forward(a16, 25, a16, -1, a16, None) == E
    assert L.spcg_mlp_forward(a16, 25, a16, 0, a16, None) == S.SPCG_OK       # B = 0: no work
    assert L.spcg_mlp_grad(a16, 25, a16, a16, 0, a16, a16, a16, None) == E  # B < 1
    assert L.spcg_mlp_grad(a16, 25, a16, a16, 4, a16, a16, None, None) == E  # no workspace
    assert L.spcg_mlp_adam(a16, a16, a16, a16, 10, 1e-3, 0, a16, None) == E  # step < 1
    assert L.spcg_mlp_adam(a16, a16, a16, a16, 0, 1e-3, 1, a16, None) == E   # P < 1
    assert L.spcg_mlp_to_bf16(None, 10, a16, None) == E
    # random maps: negative counts, NULL buffers; n = 0 is no work
    assert L.spcg_philox(None, 1, -1, None, None) == E
    assert L.spcg_philox(None, 1, 4, a16, None) == E
    assert L.spcg_philox(None, 1, 0, None, None) == S.SPCG_OK
    assert L.spcg_signs(1, -1, None, None) == E
    assert L.spcg_signs(1, 4, None, None) == E
    assert L.spcg_signs(1, 0, None, None) == S.SPCG_OK
    # context-level calls with no context or bad sizes
    info = S.Info()
    assert L.spcg_refine(None, 1e-6, 10, a16, None) == E
    assert L.spcg_export_sketch(None, 0, 1, a16, a16) == E
    assert L.spcg_export_precond(None, a16, a16, a16) == E
    assert L.spcg_features(None, a16, a16) == E
    assert L.spcg_solve_enqueue(None, a16, 1, 1) == E
    assert L.spcg_solve_result(None, ctypes.byref(info)) == E
    assert L.spcg_solve_learned(None, 1, a16, 25, a16, 1e-6, a16, ctypes.byref(info), None) == E
    assert L.spcg_solve_candidate(None, 1, 2, 1e-6, 0, a16, ctypes.byref(info)) == E
    assert L.spcg_solve_candidate(None, 1, 25, 1e-6, 0, a16, ctypes.byref(info)) == E
    # no spcg_solve_host has run in this process: nothing to trim, no CUDA call
    assert L.spcg_host_pool_trim() == S.SPCG_OK
    assert L.spcg_status_str(E) == b"SPCG_E_INVALID_ARG"


def _header_prototypes():
    """name -> (return type, [parameter types]) of every function prototype in
    include/spcg.h (comments removed; parameter names dropped)."""
    import re
    text = open(S.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\b(spcg_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3).strip()
        types = []
        if params and params != "void":
            for p in params.split(","):
                p = " ".join(p.split())
                ptr = p.count("*")
                base = re.sub(r"\bconst\b", "", p.replace("*", " "))
                words = base.split()
                # drop the parameter name (the last word) when a type precedes it
                ctype = words[0] if len(words) == 1 else " ".join(words[:-1])
                types.append((ctype, ptr))
        protos[name] = (" ".join(ret.split()), types)
    return protos


_SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
            "double": ctypes.c_double, "float": ctypes.c_float, "spcg_status": ctypes.c_int,
            "int": ctypes.c_int}


def test_binding_argument_types_match_the_header_prototypes():
    """Every binding signature has as many arguments as the header's prototype,
    a pointer where the header has a pointer and the same scalar type where it
    has a scalar, and a matching return type."""
    protos = _header_prototypes()
    assert set(protos) == set(S._SIGS)
    bad = []
    for name, (res, args) in S._SIGS.items():
        ret, params = protos[name]
        if len(params) != len(args):
            bad.append(f"{name}: {len(args)} arguments in the binding, {len(params)} in the header")
            continue
        for i, ((ctype, ptr), a) in enumerate(zip(params, args)):
            is_ptr = a is ctypes.c_void_p or a is ctypes.c_char_p or \
                isinstance(a, type) and issubclass(a, ctypes._Pointer)
            if ptr:
                if not is_ptr:
                    bad.append(f"{name} arg {i}: header {ctype} *, binding {a}")
            elif ctype in _SCALARS:
                if a is not _SCALARS[ctype]:
                    bad.append(f"{name} arg {i}: header {ctype}, binding {a}")
            else:
                bad.append(f"{name} arg {i}: unknown header type {ctype}")
        rptr = ret.count("*")
        rbase = ret.replace("*", " ").replace("const", " ").split()[-1]
        if rbase == "void" and not rptr:
            ok = res is None
        elif rptr:
            ok = res in (ctypes.c_void_p, ctypes.c_char_p)
        else:
            ok = res is _SCALARS.get(rbase)
        if not ok:
            bad.append(f"{name}: return {ret} vs {res}")
    assert not bad, bad


def test_a_c_program_links_and_calls_the_library(tmp_path):
    """The C ABI from C: a program built with gcc against include/spcg.h and
    linked to libspcg.so calls the host-only entry points (schedule, status
    string, argument errors) and gets the same answers as the binding."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "caller.c"
    src.write_text("""
#include <stdio.h>
#include "spcg.h"
int main(void) {
  spcg_schedule s;
  if (spcg_default_schedule((int64_t)1 << 20, 500, &s) != SPCG_OK) return 1;
  printf("K %d r %lld m0 %lld mK %lld a0 %d\\n", s.K, (long long)s.r, (long long)s.m[0],
         (long long)s.m[s.K - 1], s.a[0]);
  spcg_ctx* c = (spcg_ctx*)0x1;
  const int st = (int)spcg_create(NULL, NULL, 100, 5, 5, NULL, NULL, &c);
  printf("create %d null %d\\n", st, c == NULL);
  printf("str %s\\n", spcg_status_str(SPCG_E_BREAKDOWN));
  spcg_destroy(NULL);
  return 0;
}
""")
    libdir = os.path.dirname(S.LIB_PATH)
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "caller"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe),
                    "-L", libdir, "-lspcg", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = dict(zip(out[0::2], out[1::2]))
    sch = S.spcg_default_schedule(1 << 20, 500)
    assert int(got["K"]) == sch.K and int(got["r"]) == sch.r
    assert int(got["m0"]) == sch.m[0] and int(got["mK"]) == sch.m[sch.K - 1]
    assert int(got["a0"]) == sch.a[0]
    assert int(got["create"]) == S.SPCG_E_INVALID_ARG and got["null"] == "1"
    assert got["str"] == "SPCG_E_BREAKDOWN"
