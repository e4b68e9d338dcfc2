"""Collects the error summaries of the GPU-vs-oracle comparisons made by the
tests (max, p99 and mean per result kind), so that a run can report them:
with KF_PARITY_REPORT=<path> set, the session writes them there as JSON.

A comparison that fails, and a launch after which the library's device error
word is set (a bounded device wait gave up), are always recorded in full:
one JSON line per failure is appended to the file named by
KF_PARITY_FAILURE_LOG (default kf_parity_failures.jsonl in the working
directory), and the assertion message carries the worst tracks, so a failure
that does not recur can still be diagnosed."""
import json
import os

_RECORDS = []

_BRIEF_KEYS = ("n", "param", "cov", "status_mismatch", "tracks_over_bound", "worst_param",
               "worst_cov", "status_mismatch_tracks", "status_mismatch_values")


def _test_name() -> str:
    return os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]


def record(name: str, rep: dict) -> None:
    """Keep the summary of one oracle comparison (a report from
    oracle.compare.compare)."""
    _RECORDS.append({
        "test": _test_name(),
        "case": name,
        "n": rep.get("n"),
        "ok": rep.get("ok"),
        "status_equal": rep.get("status_equal"),
        "param": rep.get("param"),
        "param_by_component": rep.get("param_by_component"),
        "cov": rep.get("cov"),
    })


def failure_log_path() -> str:
    return os.environ.get("KF_PARITY_FAILURE_LOG", "kf_parity_failures.jsonl")


def _append_failure(entry: dict) -> str:
    path = failure_log_path()
    entry = {"test": _test_name(), **entry}
    try:
        with open(path, "a") as f:
            f.write(json.dumps(entry, default=str) + "\n")
    except OSError as e:  # still fail the test with the full message
        return f"(not written: {e})"
    return path


def expect_ok(name: str, rep: dict, **context) -> dict:
    """Record one comparison; when it failed, append the full report to the
    failure log and fail with its worst tracks in the message."""
    record(name, rep)
    if not rep.get("ok"):
        path = _append_failure({"case": name, "context": context, "report": rep})
        brief = {k: rep[k] for k in _BRIEF_KEYS if k in rep}
        raise AssertionError(f"{name}: GPU result outside the oracle bounds "
                             f"(full report in {path}): {json.dumps(brief, default=str)}")
    return rep


def expect_no_device_error(**context) -> None:
    """Read and clear the library's device error word; a set bit means a
    bounded device wait gave up and the launch's results are incomplete, a
    different failure from an arithmetic mismatch, so it is reported as such."""
    from paper_2401_14221_gb300 import kf

    bits = kf.kf_take_device_error()
    if bits:
        path = _append_failure({"case": "device_error", "bits": bits, "context": context})
        raise AssertionError(f"device error word {bits:#x} after the launch: a bounded device "
                             f"wait gave up (KF_DEVERR_TIMEOUT), results incomplete "
                             f"(recorded in {path})")


def dump(path: str) -> None:
    with open(path, "w") as f:
        json.dump(_RECORDS, f, indent=1)
