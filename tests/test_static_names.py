"""Every name a function of the benchmark, the entry points or the Python
binding reads is defined somewhere: a local, a parameter, an import, an
enclosing function's variable, a module global or a builtin.  The benchmark's
GPU sections only run on a GPU, so a stale name in one of them would
otherwise surface only there."""
import builtins
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ['bench.py', '__graft_entry__.py', os.path.join('paper_1411_2223_gb300', 'sq.py'),
         os.path.join('paper_1411_2223_gb300', 'build.py'), os.path.join('oracle', '__init__.py'),
         os.path.join('synth', '__init__.py')]


def undefined_names(src, name):
    table = symtable.symtable(src, name, 'exec')
    module = set(table.get_identifiers())
    found = []

    def walk(t):
        for child in t.get_children():
            if child.get_type() == 'function':
                for sym in child.get_symbols():
                    if not sym.is_referenced():
                        continue
                    if sym.is_assigned() or sym.is_parameter() or sym.is_imported() or sym.is_free():
                        continue
                    n = sym.get_name()
                    if n not in module and not hasattr(builtins, n):
                        found.append((child.get_name(), n))
            walk(child)

    walk(table)
    return found


def test_checker_finds_a_stale_name():
    src = 'def f():\n    x = 1\n    return y\n\ndef g(a):\n    return a + len([])\n'
    assert undefined_names(src, 't.py') == [('f', 'y')]


@pytest.mark.parametrize('rel', FILES)
def test_no_undefined_names(rel):
    with open(os.path.join(ROOT, rel)) as fh:
        assert undefined_names(fh.read(), rel) == []
