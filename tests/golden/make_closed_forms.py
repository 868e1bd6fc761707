"""Write the closed-form fixtures of this folder with exact rational arithmetic.

The paper prints no numerical worked example, so these fixtures are matrices
whose principal components are known exactly: X = Q diag(sigma) Z^T with Q
(M x K) and Z (N x K) having orthonormal columns with rational entries and
distinct sigma.  By Eq. 5 (the scores and loadings of X are its singular
vectors, the eigenvalues of X^T X are sigma^2), GS-PCA and NIPALS-PCA must
return lambda_k = sigma_k, P(k) = +-Z(k) and T(k) = +-sigma_k Q(k).  Nothing
here calls the oracle or the CUDA path: every stored value is the exact
product of the rational factors below.

Run from the repository root:  python tests/golden/make_closed_forms.py
"""
import os
from fractions import Fraction as F

HERE = os.path.dirname(os.path.abspath(__file__))


def matmul(A, B):
    return [[sum(A[i][t] * B[t][j] for t in range(len(B))) for j in range(len(B[0]))] for i in range(len(A))]


def transpose(A):
    return [list(r) for r in zip(*A)]


def check_orthonormal_columns(A):
    G = matmul(transpose(A), A)
    for i, row in enumerate(G):
        for j, v in enumerate(row):
            assert v == (1 if i == j else 0), (i, j, v)


def fmt(x: F) -> str:
    """Dyadic rationals as exact decimals, any other rational as p/q."""
    d = x.denominator
    return repr(float(x)) if d & (d - 1) == 0 else f"{x.numerator}/{d}"


def exact_in_float32(x: F) -> bool:
    d = x.denominator
    return d & (d - 1) == 0 and abs(x.numerator) < 2 ** 24 and d <= 2 ** 24


def write(name, Q, sigma, Z, note):
    check_orthonormal_columns(Q)
    check_orthonormal_columns(Z)
    K = len(sigma)
    S = [[sigma[i] if i == j else F(0) for j in range(K)] for i in range(K)]
    X = matmul(matmul(Q, S), transpose(Z))
    T = matmul(Q, S)
    M, N = len(X), len(X[0])
    assert all(exact_in_float32(v) for row in X for v in row), "X must be exact in FP32"
    lines = [f"# {name}: X = Q diag(sigma) Z^T, M={M} N={N} K={K}", f"# {note}",
             "# Eq. 5: lambda_k = sigma_k, P(k) = +-Z(k), T(k) = +-sigma_k Q(k) (signs free)",
             f"M {M}", f"N {N}", f"K {K}", "X"]
    lines += [" ".join(fmt(v) for v in row) for row in X]
    lines += ["lambda", " ".join(fmt(s) for s in sigma), "P"]
    lines += [" ".join(fmt(v) for v in row) for row in Z]
    lines += ["T"]
    lines += [" ".join(fmt(v) for v in row) for row in T]
    with open(os.path.join(HERE, name + ".txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


def main():
    h = F(1, 2)
    t = F(1, 3)
    # 4 x 3: Q = three columns of the 4 x 4 Hadamard matrix / 2; Z = the symmetric
    # orthogonal matrix (1/3)[[1,2,2],[2,1,-2],[2,-2,1]]; sigma = 12, 6, 3
    Q = [[h, h, h], [h, -h, h], [h, h, -h], [h, -h, -h]]
    Z = [[t, 2 * t, 2 * t], [2 * t, t, -2 * t], [2 * t, -2 * t, t]]
    sig = [F(12), F(6), F(3)]
    # Z has thirds; X = Q S Z^T does not, since every sigma is a multiple of 3
    write("closed_form_4x3", Q, sig, Z, "Q: Hadamard columns / 2; Z: (1/3)[[1,2,2],[2,1,-2],[2,-2,1]]")
    # 8 x 4 with four zero rows (a ragged zero block): Q = [H4 / 2; 0], Z = H4 / 2 with
    # its columns reordered; sigma = 16, 8, 4, 2
    H = [[h, h, h, h], [h, -h, h, -h], [h, h, -h, -h], [h, -h, -h, h]]
    Q8 = H + [[F(0)] * 4 for _ in range(4)]
    Z4 = [[row[j] for j in (2, 0, 3, 1)] for row in H]
    write("closed_form_8x4_zero_rows", Q8, [F(16), F(8), F(4), F(2)], Z4,
          "Q: [H4 / 2; 0] (rows 4-7 zero); Z: H4 / 2, columns 2, 0, 3, 1")


if __name__ == "__main__":
    main()
