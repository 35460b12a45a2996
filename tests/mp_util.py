"""Result collection for tests that run ranks as spawned processes: a rank that
dies before reporting fails the test at once instead of after the queue's
timeout, and the ranks started by the test are stopped on the way out."""
import queue
import time


def collect(q, procs, n, limit):
    """n results from q within limit seconds; fails as soon as a process has
    exited with a non-zero code."""
    got = []
    deadline = time.monotonic() + limit
    try:
        while len(got) < n:
            try:
                got.append(q.get(timeout=2))
                continue
            except queue.Empty:
                pass
            dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
            assert not dead, "a rank exited with code %s before reporting" % dead
            assert time.monotonic() < deadline, "ranks did not report within %d s" % limit
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        return got
    finally:
        for p in procs:
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
