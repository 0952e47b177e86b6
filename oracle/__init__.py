"""CPU oracle for the dedispersion search hot path -- TEST INFRASTRUCTURE ONLY.

Imported by the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py``; never by the product package.
"""
