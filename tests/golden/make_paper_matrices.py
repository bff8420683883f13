"""Write paper_matrices.txt: the integers N_i with c_ij = sqrt(15) N_i for the
Sec. 3 test matrices, from the closed form sum_k (i-1+k)(n-k) evaluated both
by brute force and by formula (they must agree).  Exact integers only."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def brute(n, i):
    return sum((i - 1 + k) * (n - k) for k in range(1, n + 1))


def formula(n, i):
    return (i - 1) * n * (n - 1) // 2 + (n - 1) * n * (n + 1) // 6


def main():
    lines = ["# n i N_i   (c_ij = sqrt(15) * N_i, Sec. 3 test matrices, 1-based i)"]
    for n in (1, 2, 7, 16, 33, 128, 1024, 4096):
        for i in sorted(v for v in {1, 2, n // 2 + 1, n} if v <= n):
            assert brute(n, i) == formula(n, i)
            lines.append("%d %d %d" % (n, i, formula(n, i)))
    with open(os.path.join(HERE, "paper_matrices.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
