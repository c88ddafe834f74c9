"""The job API (n2f_create / n2f_submit / n2f_poll / n2f_result) on the GPU: semantics, error
paths, results independent of the job mix, and what the trained network gains."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n2f():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2108_10209_gb300 import n2f as mod
    torch.cuda.set_device(0)
    return mod


def _img(h, w, seed):
    from paper_2108_10209_gb300 import synth
    clean = synth.blobs(h, w, seed=seed)
    return clean, (clean + synth.rng(seed + 1).normal(0, 0.1, (h, w))).astype(np.float32)


def test_submit_poll_result_and_errors(n2f):
    with n2f.Context() as ctx:
        _, x = _img(20, 34, 1)
        p = n2f.params(seed=2, fixed_steps=5, widths=1)
        j = ctx.submit(x, p)
        assert ctx.wait(j, 120000) == 0
        st = ctx.poll(j)
        assert st.state == n2f.N2F_DONE and st.steps == 5 and st.H == 20 and st.W == 34
        assert st.device_ms > 0 and st.t_done_ms >= st.t_start_ms
        out = ctx.result(j, x.shape)
        with pytest.raises(n2f.N2FError) as e:
            ctx.poll(j)  # collected
        assert e.value.code == n2f.N2F_ENOENT
        tr = n2f.Trainer(x, p)
        tr.run()
        assert np.array_equal(out.astype(np.float64).ravel(), tr.export(n2f.N2F_X_OUT))
        bad = x.copy()
        bad[3, 4] = np.nan
        for args in ((bad, p), (np.zeros((1, 8), np.float32), p)):
            with pytest.raises(n2f.N2FError) as e:
                ctx.submit(*args)
            assert e.value.code == n2f.N2F_EINVAL
        with pytest.raises(n2f.N2FError) as e:
            ctx.submit(x, n2f.params(precision=7))
        assert e.value.code == n2f.N2F_EINVAL


def test_odd_sizes_and_u16_input(n2f):
    from paper_2108_10209_gb300 import synth
    _, x = _img(33, 17, 5)
    q = synth.to_u16(x)
    p = n2f.params(seed=4, fixed_steps=3, widths=1)
    with n2f.Context() as ctx:
        a = ctx.submit_u16(q, p)
        b = ctx.submit((q.astype(np.float32) / np.float32(65535.0)), p)
        ctx.wait(a)
        ctx.wait(b)
        oa, ob = ctx.result(a, q.shape), ctx.result(b, q.shape)
    assert np.array_equal(oa, ob)
    ref, _ = oracle.denoise(synth.from_u16(q).astype(np.float32).astype(np.float64),
                            oracle.Params(widths=oracle.WIDTHS_W64, seed=4, fixed_steps=3))
    assert float(np.max(np.abs(oa - ref))) < 2e-3


def test_device_input_and_device_result(n2f):
    # n2f_submit_device / n2f_result_device: the job fed from device memory gives the host
    # path's result bit for bit; the binding holds the input tensor until the job is collected
    import torch
    _, x = _img(40, 36, 7)
    p = n2f.params(seed=3, fixed_steps=4, widths=1)
    with n2f.Context() as ctx:
        a = ctx.submit(x, p)
        b = ctx.submit_device(torch.from_numpy(x).cuda(), p)
        assert b in ctx._dev_inputs
        assert ctx.wait(a, 120000) == 0 and ctx.wait(b, 120000) == 0
        oa = ctx.result(a, x.shape)
        ob = torch.empty(x.shape, dtype=torch.float32, device="cuda")
        ctx.result_device(b, ob)
        assert b not in ctx._dev_inputs
    assert np.array_equal(oa, ob.cpu().numpy())


def test_results_do_not_depend_on_the_job_mix(n2f):
    # Each job runs on its own device state and stream with deterministic kernels (fixed
    # reduction orders, no atomics), so a job's output is bit-identical alone and in a mix.
    p = n2f.params(seed=9, patience=4, max_epochs=12, widths=1)
    _, x0 = _img(24, 24, 11)
    with n2f.Context() as ctx:
        j = ctx.submit(x0, p)
        ctx.wait(j)
        alone = ctx.result(j, x0.shape)
    with n2f.Context(max_slots=8) as ctx:
        others = []
        for k in range(6):
            _, xk = _img(16 + 4 * k, 40 - 2 * k, 20 + k)
            others.append((ctx.submit(xk, n2f.params(seed=k, patience=3, widths=k % 2)), xk.shape))
        j = ctx.submit(x0, p)
        for jk, shp in others:
            ctx.wait(jk)
            ctx.result(jk, shp)
        ctx.wait(j)
        mixed = ctx.result(j, x0.shape)
    assert np.array_equal(alone, mixed)


def test_cancel(n2f):
    _, x = _img(64, 64, 3)
    with n2f.Context() as ctx:
        j = ctx.submit(x, n2f.params(seed=1, patience=1000))
        assert ctx.cancel(j) == 0
        assert ctx.wait(j, 60000) == 0
        assert ctx.poll(j).state == n2f.N2F_CANCELED
        with pytest.raises(n2f.N2FError) as e:
            ctx.result(j, x.shape)
        assert e.value.code == n2f.N2F_ECANCELED


def test_budget_admission_of_the_largest_serving_size(n2f):
    """Admission against the HBM budget with 2048x2048 literal-width jobs (the largest side of
    the serving stream): under a budget of one and a half jobs' bytes the second of two jobs
    waits in the queue while the first holds the device, is admitted once the first retires,
    and both results are bit-identical to the same jobs run alone; the resident bytes never
    exceed the budget; a budget below one job's bytes refuses the job at submission."""
    import time
    from paper_2108_10209_gb300 import synth
    p = n2f.params(seed=0, fixed_steps=2)  # short runs: admission does not depend on the mode
    nb = n2f.job_bytes(2048, 2048, p)
    assert nb > (8 << 30)  # the literal-width float32 job holds more than 8 GiB
    _, noisy = synth.image_cells(2048, 2048, seed=21)
    x = noisy.astype(np.float32)
    y = np.ascontiguousarray(x[::-1])
    budget = nb + nb // 2
    with n2f.Context(hbm_budget_bytes=budget) as ctx:
        a, b = ctx.submit(x, p), ctx.submit(y, p)
        polls = 0
        while True:
            sb = ctx.poll(b).state          # b first: if a still runs afterwards, it ran here too
            sa = ctx.poll(a).state
            assert ctx.stats()["bytes_resident"] <= budget
            if sa >= n2f.N2F_DONE:
                break
            if sa == n2f.N2F_RUNNING:
                assert sb == n2f.N2F_QUEUED
                polls += 1
            time.sleep(0.0005)
        assert polls > 0
        assert ctx.wait(b, 120000) == n2f.N2F_OK and ctx.poll(b).state == n2f.N2F_DONE
        out_a, out_b = ctx.result(a, x.shape), ctx.result(b, y.shape)
    for img, out in ((x, out_a), (y, out_b)):
        assert np.array_equal(out, n2f.denoise(img, p))
    with n2f.Context(hbm_budget_bytes=nb - 1) as ctx:
        with pytest.raises(n2f.N2FError) as e:
            ctx.submit(x, p)
        assert e.value.code == n2f.N2F_ETOOBIG


def test_trained_network_gains_over_the_untrained_path(n2f):
    # The learned part: the network trained by the library's own forward/backward kernels on
    # the four checkerboard pairs denoises the full image; without training (zero steps) the
    # same path outputs the untrained network, and a 3x3 mean filter is the non-learned baseline.
    from paper_2108_10209_gb300 import synth
    clean, noisy = synth.image_cells(96, 96, sigma=25 / 255, seed=7)
    with n2f.Context() as ctx:
        j = ctx.submit(noisy, n2f.params(seed=0))
        j0 = ctx.submit(noisy, n2f.params(seed=0, fixed_steps=0))
        ctx.wait(j)
        ctx.wait(j0)
        st = ctx.poll(j)
        out, out0 = ctx.result(j, noisy.shape), ctx.result(j0, noisy.shape)
    pad = np.pad(noisy, 1, mode="reflect")
    mean3 = sum(pad[dy:dy + 96, dx:dx + 96] for dy in range(3) for dx in range(3)) / 9
    p_noisy, p_out, p_out0 = synth.psnr(noisy, clean), synth.psnr(out, clean), synth.psnr(out0, clean)
    p_mean = synth.psnr(mean3, clean)
    print(f"PSNR noisy {p_noisy:.2f}  untrained {p_out0:.2f}  mean3x3 {p_mean:.2f}  "
          f"Noise2Fast {p_out:.2f} dB (stop epoch {st.epoch})")
    assert st.stopped == 1 and st.epoch >= 101
    assert p_out > p_noisy + 3.0
    assert p_out > p_out0 + 5.0
    # and it beats the non-learned 3x3 mean filter on the same image
    assert p_out > p_mean


def test_graph_replay_matches_launch_by_launch(n2f):
    # An epoch captured once as a CUDA graph and replayed computes exactly what launching its
    # kernels one by one computes (every mutable scalar lives in device memory).
    _, x = _img(40, 36, 31)
    p = n2f.params(seed=3, patience=5, widths=1)
    outs = []
    for graphs in (False, True):
        with n2f.Context(use_graphs=graphs) as ctx:
            j = ctx.submit(x, p)
            ctx.wait(j)
            st = ctx.poll(j)
            outs.append((ctx.result(j, x.shape), st.epoch, st.steps))
    assert outs[0][1:] == outs[1][1:]
    assert np.array_equal(outs[0][0], outs[1][0])


def test_profiled_graph_replay(n2f):
    # A job that times a kernel class per launch still replays its epoch graph: the graph's
    # event-record nodes get fresh events before each replay. Results are identical to the
    # unprofiled job, and the launch count and FLOP total equal those of launch-by-launch timing.
    _, x = _img(48, 40, 33)
    p = n2f.params(seed=4, patience=4)
    ref = n2f.denoise(x, p)
    got = {}
    for kind in (n2f.N2F_K_CONV, n2f.N2F_K_CONV_WGRAD):
        for graphs in (False, True):
            with n2f.Context(profile_kernel=kind, use_graphs=graphs) as ctx:
                j = ctx.submit(x, p)
                ctx.wait(j)
                out = ctx.result(j, x.shape)
                st = ctx.stats()
            assert np.array_equal(out, ref)
            assert st["prof_launches"] > 0 and st["prof_ms"] > 0
            got[(kind, graphs)] = (st["prof_launches"], st["prof_flops"])
        assert got[(kind, False)] == got[(kind, True)]


def test_profiling_every_nth_epoch(n2f):
    # With profile_every = k only the launches of epochs 0, k, 2k, ... are timed (the epoch graph
    # is also captured without its event records and replayed on the other epochs): results are
    # unchanged, and the timed launch count is the per-epoch count times those epochs.
    _, x = _img(48, 40, 34)
    p = n2f.params(seed=4, patience=6)
    ref = n2f.denoise(x, p)
    got = {}
    for every in (1, 3):
        for graphs in (False, True):
            with n2f.Context(profile_kernel=n2f.N2F_K_CONV, use_graphs=graphs,
                             profile_every=every) as ctx:
                j = ctx.submit(x, p)
                ctx.wait(j)
                ep = ctx.poll(j).epoch
                out = ctx.result(j, x.shape)
                st = ctx.stats()
            assert np.array_equal(out, ref)
            got[(every, graphs)] = (st["prof_launches"], ep)
    full, epochs = got[(1, True)]
    assert got[(1, False)] == (full, epochs) and full % epochs == 0 and epochs > 3
    for graphs in (False, True):
        assert got[(3, graphs)] == (full // epochs * ((epochs + 2) // 3), epochs)


def test_autotuned_launches_give_identical_results(n2f):
    # The tuner only picks among launch choices that leave every result unchanged (pipeline
    # stages, CTAs per SM): tuned and untuned jobs agree bit for bit, in both forms.
    imgs = [_img(48, 40, 51)[1], _img(64, 96, 52)[1]]
    for prec in (0, 1):
        p = n2f.params(seed=6, patience=3, precision=prec)
        outs = []
        for tune in (False, True):
            with n2f.Context(autotune=tune) as ctx:
                ids = [ctx.submit(x, p) for x in imgs]
                for x, j in zip(imgs, ids):
                    assert ctx.wait(j) == 0
                outs.append([ctx.result(j, x.shape) for x, j in zip(imgs, ids)])
        for a, b in zip(*outs):
            assert np.array_equal(a, b)


def test_admission_by_hbm_budget(n2f):
    # The budget admits jobs first-in first-out while their device state fits; a job that can
    # never fit is refused at submission.
    _, x = _img(64, 64, 41)
    p = n2f.params(seed=1, fixed_steps=40)
    with n2f.Context(hbm_budget_bytes=1 << 20) as ctx:
        with pytest.raises(n2f.N2FError) as e:
            ctx.submit(x, p)
        assert e.value.code == n2f.N2F_ETOOBIG
    probe_bytes = 0
    with n2f.Context() as ctx:  # measure one job's resident bytes while it runs
        j = ctx.submit(x, p)
        while ctx.poll(j).state < n2f.N2F_DONE:
            probe_bytes = max(probe_bytes, ctx.stats()["bytes_resident"])
        ref = ctx.result(j, x.shape)
    assert probe_bytes > 0
    with n2f.Context(hbm_budget_bytes=int(probe_bytes * 1.5)) as ctx:  # one job at a time
        ids = [ctx.submit(x, p) for _ in range(3)]
        seen_queued = False
        while True:
            st = ctx.stats()
            assert st["bytes_resident"] <= int(probe_bytes * 1.5)
            seen_queued |= st["jobs_queued"] > 0 and st["jobs_running"] == 1
            if st["jobs_done"] == 3:
                break
        outs = [ctx.result(j, x.shape) for j in ids]
    assert seen_queued
    for o in outs:
        assert np.array_equal(o, ref)


@pytest.mark.parametrize("case", ["smallest 2x2", "constant", "all zeros"])
def test_degenerate_images_against_oracle(n2f, case):
    # The smallest image the method accepts (sub-images 2x1 and 1x2), a constant image (the four
    # sub-images and every target identical) and an all-zero one (BCE targets 0, the first
    # layer's output its bias alone), through the job API with the literal widths on the
    # tensor-core engine, 4 fixed steps, against the oracle's run.
    if case == "smallest 2x2":
        x = np.array([[0.2, 0.7], [0.9, 0.1]], np.float32)
    elif case == "constant":
        x = np.full((16, 24), 0.5, np.float32)
    else:
        x = np.zeros((16, 24), np.float32)
    p = n2f.params(seed=3, fixed_steps=4)
    with n2f.Context() as ctx:
        j = ctx.submit(x, p)
        assert ctx.wait(j, 120000) == n2f.N2F_OK
        out = ctx.result(j, x.shape)
    ref, _ = oracle.denoise(x.astype(np.float64), oracle.Params(seed=3, fixed_steps=4))
    assert np.all(np.isfinite(out))
    assert float(np.max(np.abs(out - ref))) < 2e-3
