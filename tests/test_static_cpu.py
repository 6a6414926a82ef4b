"""Static check of the host-side Python: every global name that a function of
bench.py, __graft_entry__.py or the package's modules reads resolves to a
module-level name or a builtin.  The GPU-only paths (the timed regions, the
nested workloads) cannot run on a host without a GPU, so a misspelt or
removed name there would otherwise surface only on the GPU."""
import builtins
import dis
import importlib
import types

import pytest

MODULES = ["bench", "__graft_entry__", "paper_2607_25272_b300.spcg",
           "paper_2607_25272_b300.inputs", "paper_2607_25272_b300.schedule_model",
           "paper_2607_25272_b300.build"]


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
