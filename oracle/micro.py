"""Python big-integer micro-oracle for tiny rings (TEST INFRASTRUCTURE ONLY).

Brute-force definitions used to pin the C core of the oracle: schoolbook
negacyclic products in Z_q[X]/(X^N + 1), direct polynomial evaluation, exact
CRT reconstruction and substitution X -> X^k.  Everything is O(N^2) Python
integers, so only small N are practical.
"""


def schoolbook_negacyclic(a, b, q):
    """a*b mod (X^N + 1, q) by the definition of the product."""
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return [x % q for x in out]


def evaluate(a, x, q):
    """a(x) mod q by Horner's rule."""
    acc = 0
    for c in reversed(a):
        acc = (acc * x + c) % q
    return acc


def substitute(a, k, q):
    """a(X^k) mod (X^N + 1, q) by expanding each monomial."""
    n = len(a)
    out = [0] * n
    for i, c in enumerate(a):
        e = (i * k) % (2 * n)
        if e < n:
            out[e] += c
        else:
            out[e - n] -= c
    return [x % q for x in out]


def crt(residues, primes):
    """The integer in [0, prod(primes)) with the given residues."""
    Q = 1
    for p in primes:
        Q *= p
    x = 0
    for r, p in zip(residues, primes):
        h = Q // p
        x += r * h * pow(h, -1, p)
    return x % Q
