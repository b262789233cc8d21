"""CPU oracle for the Blind-Match encrypted 1:N match (TEST INFRASTRUCTURE ONLY).

A plain, slow RNS-CKKS written from the paper (Sec. 2, Sec. 3.3, Algorithms 1
and 2, the compression step and Sec. 4's cost model).  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import it; it shares no
code with the GPU library.
"""
