"""Host logic of the tensor-core DFT form (build option short_dft): the
split DFT matrices that sg_dft_tc_matrices returns, decoded from their
documented core-matrix layout and pinned against numpy's real FFT.

P1 (Sec. 2, the azimuthal transform of each row): y = x D must be the
half spectrum of x packed as (X(0), X(N/2), Re X(1), Im X(1), ...).  P3: the
packed half spectrum b of a real row f times E must give N f (the inverse
transform without its 1/N, which the kernel spectra carry)."""
import numpy as np
import pytest

from paper_1509_01450_gb300 import sg

SIZES = [32, 64, 128, 256]


def decode(buf, N):
    """(D_hi, D_lo, E_hi, E_lo), each N x N indexed [input k][output j]."""
    NT, KC = min(N, 64), 32
    nct, nch = N // NT, N // KC
    j = np.arange(N)[:, None]
    k = np.arange(N)[None, :]
    t, jj, c, kk = j // NT, j % NT, k // KC, k % KC
    at = (t * nch + c) * (NT * KC) + ((jj // 8) * (KC // 4) + kk // 4) * 32 + (jj % 8) * 4 + kk % 4
    assert at.max() < N * N and len(np.unique(at)) == N * N  # a permutation of each part
    parts = buf.reshape(4, N * N)
    return [p[at].T.astype(np.float64) for p in parts]  # [k][j]


def packed_rfft(x):
    X = np.fft.rfft(x, axis=-1)
    N = x.shape[-1]
    y = np.empty(x.shape[:-1] + (N,))
    y[..., 0] = X[..., 0].real
    y[..., 1] = X[..., N // 2].real
    y[..., 2::2] = X[..., 1:N // 2].real
    y[..., 3::2] = X[..., 1:N // 2].imag
    return y


@pytest.mark.parametrize("N", SIZES)
def test_hi_parts_are_tf32_and_split_is_close(N):
    buf = sg.dft_tc_matrices(N)
    bits = buf.view(np.uint32).reshape(4, N * N)
    assert np.all(bits[0] & 0x1FFF == 0) and np.all(bits[2] & 0x1FFF == 0)  # 10 stored fraction bits
    Dh, Dl, Eh, El = decode(buf, N)
    n = np.arange(N)
    ang = 2 * np.pi * np.outer(n, n) / N
    # the exact matrices, written from their definition
    D = np.empty((N, N))
    D[:, 0], D[:, 1] = 1.0, (-1.0) ** n
    D[:, 2::2], D[:, 3::2] = np.cos(ang[:, 1:N // 2]), -np.sin(ang[:, 1:N // 2])
    E = np.empty((N, N))
    E[0, :], E[1, :] = 1.0, (-1.0) ** n
    E[2::2, :], E[3::2, :] = 2 * np.cos(ang[1:N // 2, :]), -2 * np.sin(ang[1:N // 2, :])
    assert np.max(np.abs(Dh - D)) <= 2.0 ** -11 and np.max(np.abs(Eh - E)) <= 2.0 ** -10
    assert np.max(np.abs(Dh + Dl - D)) <= 2.0 ** -23 and np.max(np.abs(Eh + El - E)) <= 2.0 ** -22


@pytest.mark.parametrize("N", SIZES)
def test_forward_matrix_gives_the_packed_half_spectrum(N):
    Dh, Dl, _, _ = decode(sg.dft_tc_matrices(N), N)
    x = np.random.default_rng(N).standard_normal((5, N))
    ref = packed_rfft(x)
    got = x @ (Dh + Dl)
    assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", SIZES)
def test_inverse_matrix_gives_N_times_the_row(N):
    _, _, Eh, El = decode(sg.dft_tc_matrices(N), N)
    f = np.random.default_rng(N + 1).standard_normal((5, N))
    got = packed_rfft(f) @ (Eh + El)
    assert np.max(np.abs(got - N * f)) <= 1e-6 * N * np.max(np.abs(f))


@pytest.mark.parametrize("N", [0, 16, 48, 512, 1024])
def test_unsupported_lengths_are_refused(N):
    with pytest.raises(sg.SgError) as e:
        sg.dft_tc_matrices(max(N, 1))
    assert e.value.status == sg.SG_ERR_UNSUPPORTED
