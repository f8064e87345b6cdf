"""Batched form (one persistent launch over many images, CUDA graph capture/replay) on
the GPU, through the C ABI.  Every image must match its one-at-a-time fbf_filter result
within the FP32 tolerance, and the oracle where the oracle is cheap."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import filters as ofl
from paper_1811_02168_gb300.synth import voronoi_image

pytestmark = pytest.mark.gpu
TOL = 5e-3
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_02168_gb300 import build
    build.build()
    from paper_1811_02168_gb300 import binding
    binding.lib()
    return binding


def _mixed_jobs(n, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        H = int(rng.integers(40, 400))
        W = int(rng.integers(40, 400))
        theta = float(rng.choice([1.0, 2.0, 5.0, 10.0]))
        sigma = float(rng.choice([10.0, 30.0, 80.0]))
        K = int(rng.choice([3, 5, 8]))
        jobs.append((H, W, theta, sigma, K, seed * 100 + i))
    return jobs


def _close(y, ref, tol=TOL):
    """Batch and lone launches differ only in the order of split-tile partial sums.  A plan with
    a poor kernel fit (e.g. K = 5 at sigma = 10, E = 3.35) can drive the Fourier denominator
    close to zero at a pixel, where the output leaves [0, 255] by orders of magnitude (1e4 in
    one test image) and a relative rounding difference shows in absolute terms: the tolerance
    scales with the output's magnitude beyond the intensity range."""
    scale = torch.clamp(ref.abs() / 255.0, min=1.0)
    return float(((y - ref).abs() / scale).max()) <= tol


def _single(B, plan, x):
    y = torch.empty_like(x)
    H, W = x.shape
    B.fbf_filter(plan.handle, x.data_ptr(), y.data_ptr(), H, W, W, torch.cuda.current_stream().cuda_stream)
    return y


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_single_launches_alone_vs_in_mix(B, autotune):
    """Each image filtered in the mix (one launch per radius class over all images) equals
    the same image filtered alone, within the FP32 tolerance."""
    jobs = _mixed_jobs(14, 3 + autotune)
    plans = {}
    xs, ys, refs = [], [], []
    batch = B.Batch(32, autotune=autotune)
    for H, W, theta, sigma, K, seed in jobs:
        key = (theta, sigma, K)
        if key not in plans:
            plans[key] = B.Plan(sigma, 255, theta, K=K)
        x = torch.from_numpy(voronoi_image(H, W, 8, 30.0, 10.0, seed=seed)).cuda()
        y = torch.full_like(x, -5.0)
        xs.append(x)
        ys.append(y)
        refs.append(_single(B, plans[key], x))
        batch.submit(plans[key], x, y)
    batch.launch()
    torch.cuda.synchronize()
    for y, ref in zip(ys, refs):
        assert float((y - ref).abs().max()) <= TOL
    batch.close()


def test_batch_against_oracle(B):
    jobs = [(70, 90, 2.0, 30.0, 5, 1), (33, 150, 5.0, 10.0, 8, 2), (120, 64, 2.0, 80.0, 3, 3)]
    batch = B.Batch(8)
    outs = []
    for H, W, theta, sigma, K, seed in jobs:
        img = voronoi_image(H, W, 8, 30.0, 10.0, seed=seed)
        plan = B.Plan(sigma, 255, theta, K=K)
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        t = batch.submit(plan, x, y)
        outs.append((img, plan, x, y, theta, sigma, K))
    batch.launch()
    batch.wait(t, 60.0)
    assert batch.poll(t) == B.FBF_DONE
    for img, plan, x, y, theta, sigma, K in outs:
        op = ofit.make_plan(sigma, 255, K=K)
        ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
        assert np.abs(y.cpu().numpy() - ref).max() <= TOL
    batch.close()


def test_graph_capture_and_replay_follow_new_input(B):
    """Capture once, replay twice with new contents in the same input buffers: each replay
    equals fbf_filter on the contents of that moment."""
    jobs = _mixed_jobs(6, 9)
    batch = B.Batch(8)
    items = []
    for H, W, theta, sigma, K, seed in jobs:
        plan = B.Plan(sigma, 255, theta, K=K)
        x = torch.from_numpy(voronoi_image(H, W, 8, 30.0, 10.0, seed=seed)).cuda()
        y = torch.empty_like(x)
        batch.submit(plan, x, y)
        items.append((plan, x, y, H, W))
    batch.capture()
    assert batch.pending() == 0
    for rep in range(2):
        for i, (plan, x, y, H, W) in enumerate(items):
            x.copy_(torch.from_numpy(voronoi_image(H, W, 8, 30.0, 10.0, seed=1000 * rep + i)).cuda())
        t = batch.replay()
        batch.wait(t, 60.0)
        for plan, x, y, H, W in items:
            assert float((y - _single(B, plan, x)).abs().max()) <= TOL
    batch.close()


def test_replay_after_a_larger_launch(B):
    """Capture a small batch, then launch a larger one through fbf_launch (its scratch must
    grow), then replay the graph: the graph keeps its own buffers, so the replay still
    equals fbf_filter image by image, and one image matches the oracle."""
    small = _mixed_jobs(3, 21)
    batch = B.Batch(16)
    items = []
    for H, W, theta, sigma, K, seed in small:
        plan = B.Plan(sigma, 255, theta, K=K)
        x = torch.from_numpy(voronoi_image(H, W, 8, 30.0, 10.0, seed=seed)).cuda()
        y = torch.empty_like(x)
        batch.submit(plan, x, y)
        items.append((plan, x, y))
    batch.capture()
    big_plan = B.Plan(30.0, 255, 5.0, K=6)
    bigs = [torch.from_numpy(voronoi_image(1500, 1400, 60, 30.0, 10.0, seed=500 + i)).cuda() for i in range(3)]
    outs = [torch.empty_like(x) for x in bigs]
    for x, y in zip(bigs, outs):
        batch.submit(big_plan, x, y)
    batch.launch()
    t = batch.replay()
    batch.wait(t, 60.0)
    for plan, x, y in items:
        assert _close(y, _single(B, plan, x))
    for x, y in zip(bigs, outs):
        assert _close(y, _single(B, big_plan, x))
    plan, x, y = items[0]
    op = ofit.make_plan(plan.sigma, 255, K=plan.K)
    ref = ofl.fourier_bf(x.cpu().numpy().astype(np.float64), plan.theta, op.c, op.T)
    assert np.abs(y.cpu().numpy() - ref).max() <= TOL
    batch.close()


def test_first_launch_on_a_non_blocking_stream(B):
    """The first launch of a fresh batch (its scratch just allocated and cleared) on a
    non-blocking stream, which is not ordered after the legacy default stream: the result
    equals fbf_filter."""
    plan = B.Plan(10.0, 255, 5.0, eps=0.01)
    xs = [torch.from_numpy(voronoi_image(700 + 13 * i, 650, 40, 30.0, 10.0, seed=40 + i)).cuda() for i in range(4)]
    ys = [torch.full_like(x, -1.0) for x in xs]
    refs = [_single(B, plan, x) for x in xs]
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    batch = B.Batch(8)
    t = 0
    for x, y in zip(xs, ys):
        t = batch.submit(plan, x, y)
    batch.launch(side)
    batch.wait(t, 60.0)
    for y, r in zip(ys, refs):
        assert _close(y, r)
    batch.close()


def test_launches_in_a_row_reuse_the_work_list_ring(B):
    """More launches than work-list slots, without synchronising in between."""
    plan = B.Plan(30.0, 255, 2.0, K=4)
    batch = B.Batch(4)
    xs = [torch.from_numpy(voronoi_image(64 + 8 * i, 80, 6, 30.0, 10.0, seed=i)).cuda() for i in range(9)]
    ys = [torch.empty_like(x) for x in xs]
    tickets = []
    for x, y in zip(xs, ys):
        tickets.append(batch.submit(plan, x, y))
        batch.launch()
    batch.wait(tickets[-1], 60.0)
    assert all(batch.poll(t) == B.FBF_DONE for t in tickets)
    for x, y in zip(xs, ys):
        assert float((y - _single(B, plan, x)).abs().max()) <= TOL
    batch.close()


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_tensor_core_forms_in_the_batch(B, form):
    """Tensor-core plans share a batch with FP32 plans (one launch per form and radius class);
    each tensor-core image equals the same image filtered alone by fbf_filter (the per-tile
    arithmetic is identical; only the order of split-tile partial sums may differ) and
    meets the 0.5 gray-level bound against the oracle."""
    prec = B.FBF_FP16_TC if form == "fp16" else B.FBF_BF16_TC
    jobs = _mixed_jobs(12, 21 if form == "fp16" else 22)
    batch = B.Batch(32)
    plans, items = {}, []
    for n, (H, W, theta, sigma, K, seed) in enumerate(jobs):
        p_here = prec if n % 3 else B.FBF_FP32
        key = (theta, sigma, K, p_here)
        if key not in plans:
            plans[key] = B.Plan(sigma, 255, theta, K=K, precision=p_here)
        img = voronoi_image(H, W, 8, 30.0, 10.0, seed=seed)
        x = torch.from_numpy(img).cuda()
        y = torch.full_like(x, -5.0)
        items.append((img, plans[key], x, y, _single(B, plans[key], x), theta, sigma, K, p_here))
        batch.submit(plans[key], x, y)
    batch.launch()
    torch.cuda.synchronize()
    for img, plan, x, y, ref, theta, sigma, K, p_here in items:
        assert _close(y, ref)
        if p_here != B.FBF_FP32 and img.size <= 60000:
            op = ofit.make_plan(sigma, 255, K=K)
            exact = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
            assert np.abs(y.cpu().numpy() - exact).max() <= 0.5
    assert B.fbf_device_errors(True) == 0
    batch.close()


def test_tensor_core_batch_graph_replay(B):
    jobs = _mixed_jobs(5, 31)
    batch = B.Batch(8)
    items = []
    for H, W, theta, sigma, K, seed in jobs:
        # K from eps = 0.01: this test is about replay, so its plans fit the kernel well (a
        # poorly fitted plan can put a pixel's denominator near zero, see _close)
        plan = B.Plan(sigma, 255, theta, eps=0.01, precision=B.FBF_BF16_TC)
        x = torch.from_numpy(voronoi_image(H, W, 8, 30.0, 10.0, seed=seed)).cuda()
        y = torch.empty_like(x)
        batch.submit(plan, x, y)
        items.append((plan, x, y, H, W))
    batch.capture()
    for rep in range(2):
        for i, (plan, x, y, H, W) in enumerate(items):
            x.copy_(torch.from_numpy(voronoi_image(H, W, 8, 30.0, 10.0, seed=500 * rep + i)).cuda())
        t = batch.replay()
        batch.wait(t, 60.0)
        for plan, x, y, H, W in items:
            assert _close(y, _single(B, plan, x))
    batch.close()


_TUNE_CHILD = r'''
import json, sys
import torch
sys.path.insert(0, sys.argv[1])
from paper_1811_02168_gb300 import binding as B
from paper_1811_02168_gb300.synth import voronoi_image
B.lib()
batch = B.Batch(8, autotune=True)
ys, refs = [], []
for theta, (H, W) in zip((2.0, 5.0, 10.0), [(300, 260), (500, 333), (700, 410)]):   # r = 6, 15, 30
    plan = B.Plan(30.0, 255, theta, K=5)
    x = torch.from_numpy(voronoi_image(H, W, 10, 30.0, 10.0, seed=H)).cuda()
    ref = torch.empty_like(x)
    B.fbf_filter(plan.handle, x.data_ptr(), ref.data_ptr(), H, W, W, torch.cuda.current_stream().cuda_stream)
    y = torch.full_like(x, -5.0)
    batch.submit(plan, x, y)
    ys.append(y)
    refs.append(ref)
batch.launch()
torch.cuda.synchronize()
print(json.dumps({"err": max(float((y - r).abs().max()) for y, r in zip(ys, refs)),
                  "device_errors": B.fbf_device_errors(True)}))
batch.close()
'''


def test_autotune_cache_file(B, tmp_path):
    """FBF_TUNE_CACHE: a first process tunes the radius classes with more than one candidate
    (r = 6, 15, 30) and appends one "key name" line per class, naming a candidate of that
    class; a second process reads the file back (with a junk line, a three-token line and a
    key paired with another class's candidate, all ignored; the last makes that class tune
    again) and filters the same images.  Both match fbf_filter within the FP32 tolerance."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = tmp_path / "child.py"
    child.write_text(_TUNE_CHILD)
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, FBF_TUNE_CACHE=str(cache))

    def run():
        out = subprocess.run([sys.executable, str(child), root], env=env, capture_output=True, text=True,
                             timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        res = json.loads(out.stdout.strip().splitlines()[-1])
        assert res["device_errors"] == 0
        assert res["err"] <= TOL
        return res

    run()
    lines = cache.read_text().split("\n")
    pairs = [ln.split() for ln in lines if ln.strip()]
    assert len(pairs) == 3 and all(len(p) == 2 for p in pairs)
    for rad, (key, name) in zip((6, 15, 30), sorted(pairs, key=lambda p: int(p[0].split("/r")[1].split("/")[0]))):
        assert f"/r{rad}/" in key and name.startswith(f"r{rad}_ty")
    key15 = next(k for k, _ in pairs if "/r15/" in k)
    # the last line for key15 names a candidate of another class: it wins the file's
    # pairing but is ignored when used, so r = 15 is tuned again and a new line appended
    cache.write_text("junk\n" + f"{key15} r15_ty96_nt512 extra\n" + "\n".join(p[0] + " " + p[1] for p in pairs) +
                     f"\n{key15} r6_ty112_nt512\n")
    run()
    last = cache.read_text().strip().split("\n")[-1].split()
    assert last[0] == key15 and last[1].startswith("r15_ty")


def test_implicit_queue_submit_and_poll(B):
    """fbf_submit / fbf_poll without a batch handle: images queued on the device's implicit
    queue are launched together at the first poll and equal fbf_filter; plans may be
    destroyed right after submitting (their parameters are copied); one image against the
    oracle."""
    jobs = _mixed_jobs(5, 33)
    items, tickets = [], []
    torch.cuda.synchronize()
    for H, W, theta, sigma, K, seed in jobs:
        plan = B.Plan(sigma, 255, theta, K=K)
        x = torch.from_numpy(voronoi_image(H, W, 8, 30.0, 10.0, seed=seed)).cuda()
        y = torch.full_like(x, -1.0)
        torch.cuda.synchronize()
        tickets.append(B.fbf_submit(plan.handle, x.data_ptr(), y.data_ptr(), H, W, W))
        items.append((H, W, theta, sigma, K, x, y))
        plan.close()
    assert len(set(tickets)) == 1          # one launch for the whole queue
    B.fbf_wait(tickets[-1], 60.0)
    assert B.fbf_poll(tickets[0]) == B.FBF_DONE
    for H, W, theta, sigma, K, x, y in items:
        assert _close(y, _single(B, B.Plan(sigma, 255, theta, K=K), x))
    H, W, theta, sigma, K, x, y = items[0]
    op = ofit.make_plan(sigma, 255, K=K)
    ref = ofl.fourier_bf(x.cpu().numpy().astype(np.float64), theta, op.c, op.T)
    assert np.abs(y.cpu().numpy() - ref).max() <= TOL
    # a second round on the same queue gets a new ticket
    H, W, theta, sigma, K, x, y = items[1]
    plan = B.Plan(sigma, 255, theta, K=K)
    y2 = torch.full_like(x, -1.0)
    t2 = B.fbf_submit(plan.handle, x.data_ptr(), y2.data_ptr(), H, W, W)
    assert t2 != tickets[0]
    while B.fbf_poll(t2) != B.FBF_DONE:
        pass
    assert _close(y2, y)   # alone in its launch: only the split-tile partial sums are cut elsewhere


def test_batch_carries_rows_for_wide_radii(B):
    """Radius classes above 15 run the work-list kernel that carries x-pass rows down each
    image's strips (one carry slot per CTA and term of the longest image): tall images of
    different K in one launch equal their lone launches, and one matches the oracle."""
    specs = [(1500, 700, 10.0, 30.0, 4), (900, 1300, 10.0, 80.0, 8), (2100, 400, 8.0, 10.0, 16),
             (600, 600, 16.0, 30.0, 3)]
    batch = B.Batch(8)
    items = []
    for i, (H, W, theta, sigma, K) in enumerate(specs):
        plan = B.Plan(sigma, 255, theta, K=K)
        x = torch.from_numpy(voronoi_image(H, W, 80, 40.0, 12.0, seed=700 + i)).cuda()
        y = torch.full_like(x, -1.0)
        batch.submit(plan, x, y)
        items.append((plan, x, y))
    batch.launch()
    torch.cuda.synchronize()
    for plan, x, y in items:
        assert _close(y, _single(B, plan, x))
    plan, x, y = items[0]
    op = ofit.make_plan(plan.sigma, 255, K=plan.K)
    ref = ofl.fourier_bf(x.cpu().numpy().astype(np.float64), plan.theta, op.c, op.T)
    assert np.abs(y.cpu().numpy() - ref).max() <= TOL
    batch.close()


def test_batch_mixes_spatial_kernels_within_a_radius_class(B):
    """FP32 batches launch each radius class once per spatial kernel (the launch's taps are a
    kernel parameter): images of one class with different theta -- r = 4, 5, 6 in the r <= 6
    class, 11, 12, 15 in the r <= 15 class, 27, 30 in the r <= 30 class (rows carried down
    the strips) -- submitted interleaved in one batch each match the oracle with their own
    theta, also after a graph replay."""
    specs = [(90, 70, 1.3, 30.0, 5), (130, 210, 3.5, 10.0, 8), (330, 90, 9.0, 30.0, 4),
             (75, 160, 1.6, 80.0, 3), (140, 100, 5.0, 30.0, 5), (300, 130, 10.0, 80.0, 6),
             (64, 64, 2.0, 10.0, 8), (110, 150, 4.0, 80.0, 4)]
    assert sorted(int(np.ceil(3 * t)) for _, _, t, _, _ in specs) == [4, 5, 6, 11, 12, 15, 27, 30]
    batch = B.Batch(16)
    items = []
    for i, (H, W, theta, sigma, K) in enumerate(specs):
        img = voronoi_image(H, W, 12, 30.0, 10.0, seed=900 + i)
        plan = B.Plan(sigma, 255, theta, K=K)
        x = torch.from_numpy(img).cuda()
        y = torch.full_like(x, -1.0)
        batch.submit(plan, x, y)
        items.append((img, plan, x, y, theta, sigma, K))
    stream = torch.cuda.current_stream()
    batch.capture(stream)
    batch.replay(stream)
    torch.cuda.synchronize()
    for img, plan, x, y, theta, sigma, K in items:
        op = ofit.make_plan(sigma, 255, K=K)
        ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
        assert np.abs(y.cpu().numpy() - ref).max() <= TOL, (theta, sigma, K)
    batch.close()


_CAND_CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1811_02168_gb300 import binding as B
from paper_1811_02168_gb300.synth import voronoi_image
from oracle import fit as ofit, filters as ofl
B.lib()
theta = float(sys.argv[2])
specs = [(700, 300, 30.0, 6), (450, 520, 10.0, 12), (300, 700, 80.0, 4)]   # K fitted at eps 0.01
batch = B.Batch(8, autotune=True)
items = []
for i, (H, W, sigma, K) in enumerate(specs):
    img = voronoi_image(H, W, 12, 30.0, 10.0, seed=5100 + i)
    plan = B.Plan(sigma, 255, theta, K=K)
    x = torch.from_numpy(img).cuda()
    y = torch.full_like(x, -5.0)
    batch.submit(plan, x, y)
    items.append((img, sigma, K, x, y))   # the device images stay alive until the launch ran
batch.launch()
torch.cuda.synchronize()
err = 0.0
for img, sigma, K, x, y in items:
    op = ofit.make_plan(sigma, 255, K=K)
    ref = ofl.fourier_bf(img.astype(np.float64), theta, op.c, op.T)
    err = max(err, float(np.abs(y.cpu().numpy() - ref).max()))
print(json.dumps({"err": err, "device_errors": B.fbf_device_errors(True)}))
batch.close()
"""

_CANDIDATES = [(6, 2.0, "r6_ty112_nt512"), (6, 2.0, "r6_ty128_nt256"),
               (15, 5.0, "r15_ty96_nt512"), (15, 5.0, "r15_ty128_nt256"),
               (24, 8.0, "r24_ty96_nt384_carry"), (24, 8.0, "r24_ty128_nt256_carry"), (24, 8.0, "r24_ty128_nt256"),
               (30, 10.0, "r30_ty96_nt384_carry"), (30, 10.0, "r30_ty128_nt256_carry"), (30, 10.0, "r30_ty128_nt256"),
               (30, 10.0, "r30_ty96_nt256"), (48, 16.0, "r48_ty64_nt128_carry"), (48, 16.0, "r48_ty64_nt128")]


@pytest.mark.parametrize("rad,theta,cand", _CANDIDATES)
def test_every_batch_candidate_matches_the_oracle(B, tmp_path, rad, theta, cand):
    """Each tile configuration of each FP32 work-list class, forced through the tune cache
    (a "key name" line for the launch's key, so the autotuner takes it without timing the
    others: no line is appended), filters three images of the class's theta, of different K
    and shape, within the FP32 tolerance of the oracle (the autotuner's trials of the other
    candidates are never compared: their outputs are rewritten).  The plans use the K that
    Algorithm 1 gives at eps = 0.01: a smaller K at sigma = 10 leaves denominators near zero,
    where errors grow with the output's size."""
    import json
    import math
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = tmp_path / "child.py"
    child.write_text(_CAND_CHILD)
    px = 700 * 300 + 450 * 520 + 300 * 700
    key = f"{torch.cuda.get_device_name(0).replace(' ', '_')}/r{rad}/px2^{int(math.floor(math.log2(px)))}/K12"
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{key} {cand}\n")
    env = dict(os.environ, FBF_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, str(child), root, str(theta)], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["device_errors"] == 0
    assert res["err"] <= TOL, res
    assert cache.read_text().strip().split("\n") == [f"{key} {cand}"]   # taken from the cache
