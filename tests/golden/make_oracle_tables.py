"""Writes tests/golden/oracle_tables_<n>loop_<id>.json.gz: the CPU oracle's
coefficient tables (oracle/integrand.py: Integrand.table_records) of a graph
whose oracle set-up takes many minutes, so that the oracle can evaluate it
without rebuilding them (the bench's CPU baseline on the four-loop workload).
Calls oracle/ only.

    python tests/golden/make_oracle_tables.py 4 23

The set-up time is stored with the tables.
"""
import gzip
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def main():
    from oracle.graphs import enumerate_graphs
    from oracle.integrand import Integrand
    n, gi = int(sys.argv[1]), int(sys.argv[2])
    t = time.perf_counter()
    I = Integrand(enumerate_graphs(n)[gi])
    setup = time.perf_counter() - t
    path = os.path.join(HERE, "oracle_tables_%dloop_%d.json.gz" % (n, gi))
    with gzip.open(path, "wt") as f:
        json.dump({"loops": n, "graph": gi, "setup_seconds": setup, "tables": I.table_records()}, f)
    print(path, "set-up %.1f s" % setup)


if __name__ == "__main__":
    main()
