"""Workload run by tests/test_gpu_checked.py in a fresh process with N2F_LIBRARY=checked: every
kernel family of the library on ragged and odd shapes, then the checked build's count of
kernel indexes found outside their tensors. Prints one JSON line; not a test module itself."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import torch
    from paper_2108_10209_gb300 import n2f, synth
    assert os.path.basename(n2f.LIB_PATH) == "libn2f_checked.so"
    torch.cuda.set_device(0)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    n2f.check_status(clear=True)
    rng = np.random.default_rng(0)
    ran = []
    for H, W in ((2, 2), (7, 9), (2, 130), (513, 257)):
        n2f.checker_gather(dev(rng.normal(size=(H, W))))
    ran.append("gather")
    for prec in (0, 1):
        for eng in (1, 2):
            for cin, cout, H, W in ((32, 32, 9, 130), (64, 32, 33, 70), (32, 64, 16, 300),
                                    (128, 256, 6, 129), (256, 256, 4, 257), (8, 16, 5, 7)):
                if eng == 2 and (cin < 32 or cout < 32):
                    continue
                x = np.maximum(rng.normal(size=(cin, H, W)), 0)
                g = rng.normal(size=(cout, H, W))
                w = rng.normal(size=(cout, cin, 3, 3)) / np.sqrt(9 * cin)
                xc, gc = n2f.pack_cg(dev(x), prec), n2f.pack_cg(dev(g), prec)
                n2f.unpack_cg(xc, cin, H, W, prec)
                n2f.conv3x3(0, xc, cin, cout, H, W, dev(w), dev(rng.normal(size=cout)),
                            precision=prec, engine=eng)
                n2f.conv3x3(1, gc, cin, cout, H, W, dev(w), mask_cg=xc, precision=prec,
                            engine=eng)
                n2f.conv3x3_wgrad(gc, xc, cin, cout, H, W, precision=prec, engine=eng)
                dw = torch.empty((cout, cin, 3, 3), device="cuda")
                db = torch.empty((cout,), device="cuda")
                n2f.conv3x3_wgrad_noalloc(gc, xc, cin, cout, H, W, dw, db, precision=prec,
                                          engine=eng)
    ran.append("op-level conv, wgrad, no-alloc wgrad")
    _, img = synth.image_cells(34, 18, seed=3)
    for widths in (0, 1):
        for prec in (0, 1):
            for eng in (0, 1):
                tr = n2f.Trainer(img, n2f.params(seed=0, widths=widths, precision=prec,
                                                 engine=eng, patience=3))
                tr.run(12)
                for what in (n2f.N2F_X_OUT, n2f.N2F_X_HIST, n2f.N2F_X_SUM):
                    tr.export(what)
                tr.close()
    ran.append("trainer runs")
    clean, noisy = synth.image_cells(40, 36, seed=4)
    with n2f.Context(group_size=2) as ctx:
        jobs = [ctx.submit(noisy, n2f.params(seed=1, fixed_steps=4)),
                ctx.submit(noisy, n2f.params(seed=1, patience=3)),
                ctx.submit(noisy, n2f.params(seed=2, patience=3)),
                ctx.submit(np.stack([noisy, clean, noisy]), n2f.params(seed=1, channels=3,
                                                                      target_channel=1,
                                                                      fixed_steps=4)),
                ctx.submit(noisy, n2f.params(seed=1, downsample=n2f.N2F_DOWN_QUAD,
                                             fixed_steps=4)),
                ctx.submit(np.stack([noisy, clean]), n2f.params(seed=1, exact=1,
                                                                fixed_steps=4)),
                ctx.submit_u16(synth.to_u16(noisy), n2f.params(seed=1, fixed_steps=4))]
        for j in jobs:
            assert ctx.wait(j, 300000) == n2f.N2F_OK
            ctx.result(j, noisy.shape)
    ran.append("job API: lockstep group, multi-channel, Quad, Exact, 16-bit")
    vol = torch.rand((5, 33, 17), device="cuda")
    n2f.max_project(vol)
    ran.append("max projection")
    fails, site = n2f.check_status(clear=True)
    print(json.dumps({"failures": fails, "first_site": site, "ran": ran}))


if __name__ == "__main__":
    main()
