"""The C-ABI library builds, loads and exports every entry point that
include/dbcsr_gb.h declares (CPU only: no compute calls without a GPU)."""
import os
import re

from paper_1910_04796_gb300 import dbcsr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^DBCSR_API\s+[\w\s\*]+?\b(dbcsr_\w+)\s*\(", txt, flags=re.M)
    return names


def test_header_declares_entry_points():
    names = declared()
    for required in ("dbcsr_create", "dbcsr_multiply", "dbcsr_get_block", "dbcsr_get_stacks", "dbcsr_release"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = dbcsr.load(build_if_missing=True)
    for name in declared():
        assert hasattr(L, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in dbcsr.SIGNATURES}
    assert set(declared()) <= bound


def test_version_string_without_gpu():
    assert "sm_103a" in dbcsr.version()


def test_init_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        return
    try:
        dbcsr.init()
    except RuntimeError as e:
        assert "no CUDA device" in str(e)
    else:
        raise AssertionError("init() must refuse to run without a GPU")


def test_every_entry_point_cites_its_passage():
    # each declaration of the boundary header is documented with the passage of
    # the paper that defines the operation, or says the paper has none
    src = open(os.path.join(ROOT, "include", "dbcsr_gb.h")).read()
    decls = re.findall(r"(/\*(?:(?!\*/).)*\*/)\s*DBCSR_API[^;]*?(dbcsr_\w+)\s*\(", src, re.S)
    assert len(decls) >= 20
    missing = [name for com, name in decls if not re.search(r"Sec\. ?[IVX]+|no counterpart", com)]
    assert not missing, missing
