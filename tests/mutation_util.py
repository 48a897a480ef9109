"""Compile a copy of an oracle module with one planted slip written into its source (for the
mutation tests: the oracle's own pins must catch each slip)."""
import importlib.util
import os

import oracle


def oracle_source(module_file):
    return open(os.path.join(os.path.dirname(oracle.__file__), module_file)).read()


def compile_variant(src, tag):
    """A new module named oracle._<tag> built from ``src``; relative imports resolve inside the
    oracle package, and the package's own modules are left untouched."""
    name = f"oracle._{tag}"
    mod = importlib.util.module_from_spec(importlib.util.spec_from_loader(name, loader=None))
    mod.__package__ = "oracle"
    exec(compile(src, f"<{tag}>", "exec"), mod.__dict__)
    return mod


def mutate(src, old, new, tag):
    if src.count(old) != 1:
        raise AssertionError(f"mutation site not found exactly once: {old}")
    return compile_variant(src.replace(old, new), tag)
