"""Writes hadamard_16x8.txt: a closed-form economic QR with exact binary inputs.

Q0 = the first 8 columns of the 16 x 16 Sylvester-Hadamard matrix divided by 4
(orthonormal columns, entries +-1/4, exact in binary), R0 = a fixed integer upper
triangular matrix with positive diagonal.  X = Q0 R0 is computed here in integer
arithmetic (X * 4 is an integer matrix), so X is exact.  By uniqueness of the
economic QR with positive diag(R) (Sec. 1's problem statement with the sign
convention diag(R) > 0), the exact factors of X are Q0 and R0.

Run:  python tests/golden/make_hadamard_case.py   (uses no code from oracle/ or
the CUDA path).
"""
import os


def sylvester(n):
    h = [[1]]
    while len(h) < n:
        h = [row + row for row in h] + [row + [-v for v in row] for row in h]
    return h


def main():
    m, n = 16, 8
    h = sylvester(m)
    r0 = [[0] * n for _ in range(n)]
    diag = [8, 7, 6, 5, 4, 3, 2, 1]
    off = [3, -2, 1, -1, 2, -3, 1, 2, -1, 3, -2, 1, 1, -1, 2, -2, 3, 1, -3, 2, -1, 1, 2, -2, 1, -1, 3, 2]
    t = 0
    for i in range(n):
        r0[i][i] = diag[i]
        for j in range(i + 1, n):
            r0[i][j] = off[t % len(off)]
            t += 1
    # 4 X = H[:, :8] R0 (integers)
    x4 = [[sum(h[r][k] * r0[k][j] for k in range(n)) for j in range(n)] for r in range(m)]
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "hadamard_16x8.txt"), "w") as f:
        f.write("# Closed-form economic QR X = Q0 R0 (Sec. 1 problem statement, diag(R) > 0).\n")
        f.write("# Q0 = Sylvester-Hadamard H16[:, :8] / 4; X = X4 / 4 exactly.\n")
        f.write("# Written by tests/golden/make_hadamard_case.py (integer arithmetic).\n")
        f.write(f"m {m} n {n}\n")
        f.write("R0\n")
        for row in r0:
            f.write(" ".join(str(v) for v in row) + "\n")
        f.write("X4\n")
        for row in x4:
            f.write(" ".join(str(v) for v in row) + "\n")


if __name__ == "__main__":
    main()
