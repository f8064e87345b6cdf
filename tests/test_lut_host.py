"""Lookup table of K* and T* (Section II after Algorithm 1, Fig. 2), host side through the C ABI.

Pins: table entries equal the FP64 oracle's Algorithm 1 at grid points; lookups at grid nodes
return the entries; the paper's stated trends (K* falls and T* rises with sigma, both rise
with log(1/eps)); and its accuracy claim, a PSNR loss of at most 1-2 dB for interpolated
(K, T) against Algorithm 1 at the same off-grid (sigma, eps), measured with the oracle's
brute force of eq. (1)."""
import numpy as np
import pytest

from oracle import filters as ofl
from oracle import fit as ofit
from paper_1811_02168_gb300 import binding as B
from paper_1811_02168_gb300.synth import voronoi_image

SIGMAS = [float(s) for s in range(10, 85, 5)]        # 10, 15, ..., 80
EPS = [0.1, 0.05, 0.02, 0.01, 0.005, 0.002, 0.001]


@pytest.fixture(scope="module")
def lut():
    return B.Lut(255, SIGMAS, EPS)


@pytest.mark.parametrize("i,j", [(8, 3), (14, 5), (4, 0)])
def test_entries_are_algorithm1(lut, i, j):
    K, T, _, _ = ofit.algorithm1(ofit.kernel_samples(SIGMAS[i], 255), 255, EPS[j])
    assert lut.entry(i, j) == (K, T)


def test_lookup_at_nodes_and_midpoints(lut):
    for i, s in enumerate(SIGMAS):
        for j, e in enumerate(EPS):
            assert lut.lookup(s, e) == lut.entry(i, j)
    # halfway in sigma at a node of eps: the rounded mean of the two neighbours
    K0, T0 = lut.entry(1, 2)
    K1, T1 = lut.entry(2, 2)
    K, T = lut.lookup(17.5, EPS[2])
    assert abs(K - 0.5 * (K0 + K1)) <= 0.5 and abs(T - 0.5 * (T0 + T1)) <= 0.5
    # halfway in log(1/eps) at a node of sigma
    Ka, Ta = lut.entry(8, 1)
    Kb, Tb = lut.entry(8, 2)
    K, T = lut.lookup(50.0, float(np.sqrt(EPS[1] * EPS[2])))
    assert abs(K - 0.5 * (Ka + Kb)) <= 0.5 and abs(T - 0.5 * (Ta + Tb)) <= 0.5


def test_trends_of_the_table(lut):
    Ks = np.array([[lut.entry(i, j)[0] for j in range(len(EPS))] for i in range(len(SIGMAS))])
    Ts = np.array([[lut.entry(i, j)[1] for j in range(len(EPS))] for i in range(len(SIGMAS))])
    assert np.all(np.diff(Ks, axis=0) <= 0)      # K* does not grow with sigma
    assert np.all(np.diff(Ks, axis=1) >= 0)      # K* and T* grow as eps falls
    assert np.all(np.diff(Ts, axis=1) >= 0)
    # T* grows with sigma at a fixed order (it steps back where K* drops by one)
    same_k = np.diff(Ks, axis=0) == 0
    assert np.all(np.diff(Ts, axis=0)[same_k] >= 0)
    assert Ts[-1].min() > Ts[0].max()


@pytest.mark.parametrize("sigma,eps", [(27.5, 0.03), (42.0, 0.007), (66.0, 0.05), (13.0, 0.003), (71.0, 0.0015)])
def test_psnr_loss_of_interpolated_parameters(lut, sigma, eps):
    theta = 2.0
    img = voronoi_image(128, 128, 12, 40.0, 10.0, seed=77).astype(np.float64)
    ref = ofl.brute_bf(img, theta, sigma)
    p_lut = lut.plan(sigma, eps, theta)
    p_opt = B.Plan(sigma, 255, theta, eps=eps)
    psnr = {}
    for name, p in (("lut", p_lut), ("alg1", p_opt)):
        psnr[name] = ofl.psnr(ofl.fourier_bf(img, theta, np.asarray(p.c), p.T), ref)
    assert psnr["alg1"] - psnr["lut"] <= 2.0, psnr
    assert (p_lut.K, p_lut.T) == lut.lookup(sigma, eps)


def test_lut_plan_fits_only_c(lut):
    # the plan keeps the looked-up (K, T) and its coefficients are the least squares at that T
    K, T = lut.lookup(33.0, 0.02)
    p = lut.plan(33.0, 0.02, 3.0)
    assert (p.K, p.T) == (K, T)
    E, c = ofit.kernel_error(K, T, ofit.kernel_samples(33.0, 255), 255)
    assert np.allclose(p.c, c, rtol=1e-9, atol=1e-12)


def test_save_load_and_errors(lut, tmp_path):
    path = str(tmp_path / "k_t.lut")
    lut.save(path)
    back = B.Lut(path=path)
    for i in range(len(SIGMAS)):
        for j in range(len(EPS)):
            assert back.entry(i, j) == lut.entry(i, j)
    assert back.lookup(42.0, 0.02) == lut.lookup(42.0, 0.02)
    bad = tmp_path / "bad.lut"
    for text in ("fbf-lut 1\n255 2 2\n10\n",                                     # truncated
                 "fbf-lut 1\n2147483647 2 2\n10\n20\n0.1\n0.01\n1 1\n1 1\n1 1\n1 1\n",  # R too large
                 "fbf-lut 1\n255 2 2\n-10\n20\n0.1\n0.01\n1 1\n1 1\n1 1\n1 1\n",       # sigma <= 0
                 "fbf-lut 1\n255 2 2\n10\n20\n0.1\n0.01\n1 1\n0 1\n1 1\n1 1\n"):       # K = 0
        bad.write_text(text)
        with pytest.raises(B.FbfError) as ei:
            B.Lut(path=str(bad))
        assert ei.value.code == B.FBF_EINVAL
    good = "fbf-lut 1\n255 2 2\n10\n20\n0.1\n0.01\n1 1\n1 1\n1 1\n1 1\n"
    bad.write_text(good)
    assert B.Lut(path=str(bad)).entry(1, 1) == (1, 1)
    with pytest.raises(B.FbfError) as ei:
        lut.lookup(5.0, 0.01)                      # sigma below the grid
    assert ei.value.code == B.FBF_EUNSUPPORTED
    with pytest.raises(B.FbfError) as ei:
        lut.lookup(20.0, 0.0005)                   # eps beyond the grid
    assert ei.value.code == B.FBF_EUNSUPPORTED
    with pytest.raises(B.FbfError) as ei:
        B.Lut(255, [10.0, 10.0], [0.1, 0.01])      # sigmas not increasing
    assert ei.value.code == B.FBF_EINVAL
    with pytest.raises(B.FbfError) as ei:
        B.Lut(255, [10.0, 20.0], [0.01, 0.1])      # eps not decreasing
    assert ei.value.code == B.FBF_EINVAL
