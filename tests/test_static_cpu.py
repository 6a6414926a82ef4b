"""Static checks of the host-side Python: in bench.py, __graft_entry__.py, the
package's modules and the GPU test modules every global name a function reads
resolves, every attribute read through an imported module of this repository
exists, and every call into the binding matches its signature.  The GPU-only
paths (the timed regions, the nested workloads, the GPU tests) cannot run on
a host without a GPU, so such a slip would otherwise surface only on the GPU."""
import ast
import builtins
import dis
import importlib
import types

import pytest

GPU_TESTS = ["test_gpu_batched", "test_gpu_configs", "test_gpu_learned", "test_gpu_mixed",
             "test_gpu_parity", "test_gpu_resid", "test_gpu_variants", "test_zz_no_alloc"]
MODULES = ["bench", "__graft_entry__", "paper_2607_25272_b300.spcg",
           "paper_2607_25272_b300.inputs", "paper_2607_25272_b300.schedule_model",
           "paper_2607_25272_b300.build"] + GPU_TESTS
CALLERS = ["bench.py", "__graft_entry__.py", "paper_2607_25272_b300/schedule_model.py"] + \
    [f"tests/{m}.py" for m in GPU_TESTS]


def _functions(mod):
    for name, obj in vars(mod).items():
        if isinstance(obj, types.FunctionType) and obj.__module__ == mod.__name__:
            yield name, obj.__code__
        elif isinstance(obj, type) and obj.__module__ == mod.__name__:
            for k, v in vars(obj).items():
                f = v.__func__ if isinstance(v, (staticmethod, classmethod)) else v
                if isinstance(f, types.FunctionType):
                    yield f"{name}.{k}", f.__code__
                elif isinstance(v, property):
                    for acc in (v.fget, v.fset, v.fdel):
                        if acc is not None:
                            yield f"{name}.{k}", acc.__code__


def _globals_read(code):
    for ins in dis.get_instructions(code):
        if ins.opname == "LOAD_GLOBAL":
            yield ins.argval
    for c in code.co_consts:
        if isinstance(c, types.CodeType):
            yield from _globals_read(c)


@pytest.mark.parametrize("modname", MODULES)
def test_every_global_name_resolves(modname):
    mod = importlib.import_module(modname)
    known = set(vars(mod)) | set(dir(builtins))
    missing = {}
    for fname, code in _functions(mod):
        bad = sorted(set(n for n in _globals_read(code) if n not in known))
        if bad:
            missing[fname] = bad
    assert not missing, missing


def _module_aliases(tree):
    """alias -> module name for every `from X import Y as Z` / `import X as Z`."""
    out = {}
    for node in ast.walk(tree):
        if isinstance(node, ast.ImportFrom) and node.module:
            for a in node.names:
                out[a.asname or a.name] = f"{node.module}.{a.name}"
        elif isinstance(node, ast.Import):
            for a in node.names:
                out[a.asname or a.name] = a.name
    return out


@pytest.mark.parametrize("path", CALLERS)
def test_attributes_of_the_binding_and_oracle_modules_exist(path):
    """Every `alias.name` read through an imported module of this repository
    (the binding, the schedule model, the generators, the oracle) names an
    attribute that module has."""
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    tree = ast.parse(open(os.path.join(root, path)).read())
    aliases = {k: v for k, v in _module_aliases(tree).items()
               if v.startswith(("paper_2607_25272_b300.", "oracle."))}
    missing = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name) \
                and node.value.id in aliases:
            modname = aliases[node.value.id]
            try:
                mod = importlib.import_module(modname)
            except ImportError:
                continue        # a function or class imported by name, not a module
            if not hasattr(mod, node.attr):
                missing.append(f"{node.value.id}.{node.attr} (line {node.lineno})")
    assert not missing, missing


@pytest.mark.parametrize("path", CALLERS)
def test_methods_called_on_solver_objects_exist(path):
    """A name bound to `S.Solver(...)` or `S.Batch(...)` (S the binding
    module) is only used with attributes that class defines."""
    import os

    from paper_2607_25272_b300 import spcg as S
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    tree = ast.parse(open(os.path.join(root, path)).read())
    classes = {"Solver": S.Solver, "Batch": S.Batch}
    missing, checked = [], 0
    for fn in ast.walk(tree):
        if not isinstance(fn, (ast.FunctionDef, ast.Module)):
            continue
        bound = {}
        for node in ast.walk(fn):
            if isinstance(node, ast.Assign) and isinstance(node.value, ast.Call) \
                    and isinstance(node.value.func, ast.Attribute) \
                    and isinstance(node.value.func.value, ast.Name) \
                    and node.value.func.value.id == "S" and node.value.func.attr in classes:
                for t in node.targets:
                    if isinstance(t, ast.Name):
                        bound[t.id] = classes[node.value.func.attr]
        for node in ast.walk(fn):
            if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name) \
                    and node.value.id in bound:
                checked += 1
                cls = bound[node.value.id]
                if not hasattr(cls, node.attr) and node.attr not in _instance_attrs(cls):
                    missing.append(f"{node.value.id}.{node.attr} (line {node.lineno})")
    assert not missing, missing


def _instance_attrs(cls):
    """Attributes that the class's __init__ assigns on self."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(cls))
    names = set()
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name) \
                and node.value.id == "self" and isinstance(node.ctx, ast.Store):
            names.add(node.attr)
    return names


def _call_shape(call):
    """(number of positional arguments, keyword names) or None when the call
    unpacks *args or **kwargs."""
    if any(isinstance(a, ast.Starred) for a in call.args) or any(k.arg is None for k in call.keywords):
        return None
    return len(call.args), [k.arg for k in call.keywords]


@pytest.mark.parametrize("path", CALLERS)
def test_calls_into_the_binding_match_its_signatures(path):
    """Every call `S.f(...)` of a binding function, `S.Solver(...)`,
    `S.Batch(...)` and `obj.method(...)` on such objects passes arguments
    that the Python signature accepts (number of positional arguments and
    keyword names)."""
    import inspect
    import os

    from paper_2607_25272_b300 import spcg as S
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    tree = ast.parse(open(os.path.join(root, path)).read())
    classes = {"Solver": S.Solver, "Batch": S.Batch}
    bad, checked = [], 0

    def check(fn, call, skip_self):
        nonlocal checked
        shape = _call_shape(call)
        if shape is None:
            return
        try:
            sig = inspect.signature(fn)
        except (TypeError, ValueError):
            return
        npos, kws = shape
        args = [None] * (npos + (1 if skip_self else 0))
        try:
            sig.bind(*args, **{k: None for k in kws})
            checked += 1
        except TypeError as e:
            bad.append(f"line {call.lineno}: {e}")

    for fn in ast.walk(tree):
        if not isinstance(fn, ast.FunctionDef):
            continue
        bound = {}
        for node in ast.walk(fn):
            if isinstance(node, ast.Assign) and isinstance(node.value, ast.Call) \
                    and isinstance(node.value.func, ast.Attribute) \
                    and isinstance(node.value.func.value, ast.Name) \
                    and node.value.func.value.id == "S" and node.value.func.attr in classes:
                for t in node.targets:
                    if isinstance(t, ast.Name):
                        bound[t.id] = classes[node.value.func.attr]
        for node in ast.walk(fn):
            if not (isinstance(node, ast.Call) and isinstance(node.func, ast.Attribute)
                    and isinstance(node.func.value, ast.Name)):
                continue
            owner, attr = node.func.value.id, node.func.attr
            if owner == "S" and hasattr(S, attr) and callable(getattr(S, attr)):
                target = getattr(S, attr)
                if isinstance(target, type) and attr in classes:
                    check(target.__init__, node, skip_self=True)
                elif inspect.isfunction(target):
                    check(target, node, skip_self=False)
            elif owner in bound and inspect.isfunction(getattr(bound[owner], attr, None)):
                check(getattr(bound[owner], attr), node, skip_self=True)
    assert not bad, bad
