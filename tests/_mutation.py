"""Runner of the mutation checks: a copy of a package, one planted mistake
at a time, rebuilt if it has a build step, and pin files run against the
copy in a process of their own.  Every mistake must make a pin fail (pytest
exit code 1: a crash, a hang or a broken run does not count) and the
unmutated copy must pass."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def mutate(src, name, old, new, nth=0):
    """src with the nth occurrence (from 0) of old replaced by new."""
    k = -1
    for _ in range(nth + 1):
        k = src.find(old, k + 1)
        assert k >= 0, "not in the source: " + name
    return src[:k] + new + src[k + len(old):]


def _run(work, package, files, test_files, build):
    d = os.path.join(work, package)
    os.makedirs(d)
    for name, src in files.items():
        with open(os.path.join(d, name), "w") as f:
            f.write(src)
    env = dict(os.environ, PYTHONPATH=work + os.pathsep + ROOT, PYTHONDONTWRITEBYTECODE="1")
    if build:
        subprocess.run([sys.executable, "-c", build], cwd=work, env=env, check=True, capture_output=True,
                       timeout=300)
    code = ("import os, sys, %s as pkg\n"
            "assert os.path.dirname(pkg.__file__) == %r, pkg.__file__\n"
            "import pytest\n"
            "sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', '-m', 'not gpu'] + %r))\n"
            % (package, d, [os.path.join(ROOT, f) for f in test_files]))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=work, env=env, capture_output=True, text=True,
                           timeout=180)
    except subprocess.TimeoutExpired:
        return None, "no result within 180 s"
    return r.returncode, r.stdout[-400:] + r.stderr[-400:]


def check_all(tmp_path, package, base, jobs, test_files, build=None):
    """base: {file name: source} of the package copy; jobs: [(what the
    mistake is, {file name: mutated source})]."""
    runs = [("control", {})] + list(jobs)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda k: _run(str(tmp_path / ("m%03d" % k)), package, dict(base, **runs[k][1]),
                                         test_files, build), range(len(runs))))
    rc0, out0 = res[0]
    assert rc0 == 0, "the unmutated copy fails its pins:\n" + out0
    survived = [(runs[k][0], res[k][1]) for k in range(1, len(runs)) if res[k][0] != 1]
    assert not survived, "mistakes no pin catches (or that broke the run): %s" % survived
