"""Assertion helper of the GPU parity tests: prints every measured error with
its bar (visible with `pytest -s`), so that the errors behind each bar can be
recorded, then asserts it."""
import os


def check(err, bar, what=""):
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    print(f"PARITY {test} {what} err={err:.3e} bar={bar:.1e}", flush=True)
    assert err <= bar, f"{test} {what}: error {err:.3e} above the bar {bar:.1e}"
