"""bench.py and __graft_entry__.py call the package only through names it exports (CPU)."""

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_package_name_used_by_the_bench_exists():
    import paper_2503_21176_gb300 as qg

    for script in ("bench.py", "__graft_entry__.py"):
        with open(os.path.join(ROOT, script)) as fh:
            names = set(re.findall(r"\bqg\.([A-Za-z_][A-Za-z0-9_]*)", fh.read()))
        missing = sorted(n for n in names if n != "_lib" and not hasattr(qg, n))
        assert not missing, f"{script} uses qg.{missing}"
