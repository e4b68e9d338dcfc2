"""Collects the error summaries of the GPU-vs-oracle comparisons made by the
tests (max, p99 and mean per result kind), so that a run can report them:
with KF_PARITY_REPORT=<path> set, the session writes them there as JSON."""
import json
import os

_RECORDS = []


def record(name: str, rep: dict) -> None:
    """Keep the summary of one oracle comparison (a report from
    oracle.compare.compare)."""
    _RECORDS.append({
        "test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0],
        "case": name,
        "n": rep.get("n"),
        "ok": rep.get("ok"),
        "status_equal": rep.get("status_equal"),
        "param": rep.get("param"),
        "param_by_component": rep.get("param_by_component"),
        "cov": rep.get("cov"),
    })


def dump(path: str) -> None:
    with open(path, "w") as f:
        json.dump(_RECORDS, f, indent=1)
