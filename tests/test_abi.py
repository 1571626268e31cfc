"""The C-ABI library loads and exports every function include/st.h declares."""
import re
import subprocess
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|size_t|char|uint\w+|float)\s*\**\s*(st_\w+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ("st_scene_create", "st_build_tiles", "st_trace", "st_scene_update_prims", "st_prep_tree"):
        assert n in names


def test_library_exports_every_declared_symbol(stlib):
    out = subprocess.run(["nm", "-D", "--defined-only", str(stlib.LIB_PATH)], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = declared_functions() - exported
    assert not missing, missing
    for n in declared_functions():
        getattr(stlib.lib(), n)


def test_version_string(stlib):
    assert "sm_103a" in stlib.st_version()
