"""Standalone launches of the centre move's hot kernels, for profilers.

    python -m paper_2511_05719_gb300.kernel_driver [--batch 152] [--n 256] [--m 9344]

runs, twice each: the FP64 eigensolver on `--batch` bond Gram matrices of
size n (the MIXED runs' route: ttn_eig_gram route 3, kept rank <= 128,
floor 1e-6) and the exact tensor-core Gram matrix of one m x n complex64 bond
matrix (ttn_gram_exact).  The Gram matrices are G = X^H X with X a 2n x n
complex Gaussian matrix whose columns are scaled by logspace(0, -6), a
decaying spectrum like a bond's Schmidt values; m = 9344 is the mean row
count of an n = 256 move at d = 7, chi = 128.  Everything runs on the
current CUDA device through the package's public calls.
"""
import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--batch", type=int, default=152)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--m", type=int, default=9344)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    import torch
    from . import eig_gram, gram_exact
    torch.manual_seed(a.seed)
    n = a.n
    X = torch.randn(a.batch, 2 * n, n, dtype=torch.complex128, device="cuda")
    X = X * torch.logspace(0, -6, n, dtype=torch.float64, device="cuda")
    G = X.conj().transpose(1, 2) @ X
    G = 0.5 * (G + G.conj().transpose(1, 2))
    for _ in range(2):
        V, s, k = eig_gram(G, kcap=min(n, 128), route="mixed", eps_keep=1e-6)
    torch.cuda.synchronize()
    M = torch.randn(a.m, n, dtype=torch.complex64, device="cuda")
    for _ in range(2):
        gram_exact(M)
    torch.cuda.synchronize()
    print("kept rank %d, largest singular value %.6g" % (int(k[0]), float(s[0, 0])))


if __name__ == "__main__":
    main()
