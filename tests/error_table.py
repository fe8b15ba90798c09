"""Markdown table of the errors the GPU tests measured against the oracle.

The tests record every comparison in a JSON log when PSPS_ERROR_LOG names a
file (tests/conftest.py): named records (quantity, error, bound) and the
relative L2 error of every rel_l2 call, under the test's id.  This prints,
per test, the largest error of each quantity and its bound:

    PSPS_ERROR_LOG=errors.json python -m pytest tests -m gpu
    python tests/error_table.py errors.json [more.json ...]
"""
from __future__ import annotations

import json
import sys


def rows(paths):
    for p in paths:
        yield from json.load(open(p))


def table(paths) -> str:
    best: dict = {}
    for r in rows(paths):
        test = r["test"].split("::")[-1]
        key = (test, r["quantity"])
        e = float(r["error"])
        if key not in best or e > best[key][0]:
            best[key] = (e, r.get("bound"), r.get("ratio"))
    out = ["| test | quantity | max error | bound | error / bound |", "|---|---|---|---|---|"]
    for (test, q), (e, b, ratio) in sorted(best.items()):
        if ratio is None and b:
            ratio = e / b if b else None
        out.append(f"| {test} | {q} | {e:.2e} | {'' if b is None else f'{b:.2e}'} | "
                   f"{'' if ratio is None else f'{ratio:.3f}'} |")
    return "\n".join(out)


if __name__ == "__main__":
    print(table(sys.argv[1:]))
