"""The design notes' file map points at files that exist, and every entry point the C header
declares is named there or in the README (documentation kept in step with the code)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _read(name):
    with open(os.path.join(ROOT, name)) as fh:
        return fh.read()


def test_file_map_paths_exist():
    text = _read("DESIGN.md")
    sec = text[text.index("## 11. Which file covers which part of the survey"):]
    sec = sec[:sec.index("\n## ", 5)] if "\n## " in sec[5:] else sec
    missing = []
    for path in re.findall(r"`([A-Za-z0-9_./]+\.(?:py|cu|cuh|h|c|md|txt))`", sec):
        cands = [path, os.path.join("paper_2305_09910_gb300", path), os.path.join("paper_2305_09910_gb300", "csrc", path),
                 os.path.join("tests", path), os.path.join("oracle", path)]
        if not any(os.path.exists(os.path.join(ROOT, c)) for c in cands):
            missing.append(path)
    assert not missing, missing


def test_header_entry_points_are_documented():
    header = _read("include/lbm.h")
    names = sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", header)))
    docs = _read("DESIGN.md") + _read("README.md")
    undocumented = [n for n in names if n not in docs]
    assert not undocumented, undocumented
