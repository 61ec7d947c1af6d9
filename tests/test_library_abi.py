"""The C-ABI library builds, loads without a GPU and exports every symbol
declared in include/pluqmodp.h (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "pluqmodp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*)\s+(\w+)\s*\(", text, flags=re.M)))


def test_header_declares_boundary():
    names = _declared()
    for required in ["pluq_modp", "echelon_modp", "rank_profile_modp", "pluq_modp_batched",
                     "fgemm_modp", "pluq_create", "pluq_destroy"]:
        assert required in names


def test_library_loads_and_exports_all_symbols():
    from paper_1402_3501_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), f"missing export {name}"
    from paper_1402_3501_gb300 import binding
    assert sorted(binding.SYMBOLS) == _declared()
    f = lib.pluq_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(-2) == b"p is not prime"


def test_status_codes_match_binding():
    from paper_1402_3501_gb300 import binding
    text = open(os.path.join(ROOT, "include", "pluqmodp.h")).read()
    codes = {int(v): k for k, v in re.findall(r"#define (PLUQ_(?:OK|ERR_\w+))\s+(-?\d+)", text)}
    assert set(codes) == set(binding.STATUS)


def test_options_match_binding():
    """Every PLUQ_OPT_* code of the header has the binding's name for it, and the
    binding names no option the header lacks; leaf kinds cover the documented range."""
    from paper_1402_3501_gb300 import binding
    text = open(os.path.join(ROOT, "include", "pluqmodp.h")).read()
    opts = {k.lower(): int(v) for k, v in re.findall(r"#define PLUQ_OPT_(\w+)\s+(\d+)", text)}
    assert opts == binding.Context.OPTIONS
    lo, hi = (int(x) for x in re.search(r"PLUQ_OPT_LEAF_KIND\s+leaf kernel \[(\d+), (\d+)\]",
                                        text).groups())
    assert sorted(binding.Context.LEAF_KINDS) == list(range(lo, hi + 1))
