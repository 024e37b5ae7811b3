"""The C-ABI library builds, loads, and exports every entry point that
include/mwj.h declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_1905_13376_gb300 import binding

HDR_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for fn in os.listdir(HDR_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HDR_DIR, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mwj_\w+)\s*\(", text, re.M):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("mwj_join3_linear", "mwj_join3_cyclic", "mwj_cascade_join",
                 "mwj_workspace_size", "mwj_stream_status", "mwj_create", "mwj_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    raw = ctypes.CDLL(binding.lib_path())
    for name in declared_functions():
        assert hasattr(raw, name), f"{name} declared in include/ but not exported"
    assert lib.mwj_version().decode().startswith("mwj")


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(binding._SIGS)


def test_null_arguments_rejected_without_gpu():
    lib = binding.load()
    assert lib.mwj_create(None, None) == binding.MWJ_ERR_INVALID_ARG
    assert lib.mwj_destroy(None) == binding.MWJ_ERR_INVALID_ARG
    assert lib.mwj_stream_status(None, None) == binding.MWJ_ERR_INVALID_ARG
