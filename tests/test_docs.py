"""The design notes stay in step with the sources: every CUDA kernel in csrc/
appears in the kernel inventory, and every call the header declares appears
in the notes (CPU only)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def kernels():
    names = set()
    for f in glob.glob(os.path.join(ROOT, "paper_2511_02510_gb300", "csrc", "*.cu")):
        text = open(f).read()
        for m in re.finditer(r"__global__", text):
            k = re.search(r"\b(k_[a-z0-9_]+)\s*\(", text[m.end():m.end() + 400])
            if k:
                names.add(k.group(1))
    return names


def test_every_kernel_is_in_the_inventory():
    design = open(os.path.join(ROOT, "DESIGN.md")).read()
    inventory = design[design.index("## 15. Kernel inventory"):]
    ks = kernels()
    assert len(ks) > 40
    missing = sorted(k for k in ks if f"`{k}" not in inventory and f" {k}" not in inventory)
    assert not missing, missing


def test_every_declared_call_is_in_the_notes():
    from test_abi import declared_functions
    notes = open(os.path.join(ROOT, "DESIGN.md")).read() + open(os.path.join(ROOT, "README.md")).read()
    internal = {"lv_version", "lv_last_error", "lv_launch_count"}
    # the size queries are documented together, as the `*_workspace_size` query of their call
    missing = sorted(n for n in declared_functions()
                     if n not in notes and n not in internal and not n.endswith("_workspace_size"))
    assert not missing, missing
