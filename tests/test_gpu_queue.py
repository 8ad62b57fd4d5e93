"""Persistent job queue: one launch over ciphertexts of two rings (N = 2^12 and 2^13, different
prime chains) at uneven levels, bit for bit against the oracle's HADD / subtraction / HMULPLAIN;
dependent jobs (including a serial chain whose tiles wait on one another); the hazard and
argument checks; the bounded wait on an external flag, released and never released."""
import pytest

from oracle.ckks import Plaintext
from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rings(gpu):
    a = Pair(gpu, 12, 5, 1, 1, seed=(0x9A, 1, 1, 1), relin=False, gpu_keys=False)
    b = Pair(gpu, 13, 6, 1, 1, mid_bits=45, seed=(0x9B, 2, 2, 2), relin=False, gpu_keys=False)
    yield a, b
    a.close()
    b.close()


def operands(p, lvl, tag):
    o = p.orc
    x = o.encrypt_sk(o.encode(synth.slots(tag, 64), level=lvl), tag)
    y = o.encrypt_sk(o.encode(synth.slots(tag + 1, 64), level=lvl), tag + 1)
    pt = o.encode(synth.slots(tag + 2, 64), level=p.orc.L)  # above the ciphertext: leading limbs
    return x, y, pt


def test_mixed_rings_and_levels_one_launch(rings):
    pf = rings[0].pft
    jobs, checks = [], []
    tag = 100
    for lvl in (1, 2, 3, 4, 5, 6):  # interleave the two rings
        for p in rings:
            if lvl > p.orc.L:
                continue
            o = p.orc
            x, y, pt = operands(p, lvl, tag)
            tag += 10
            gx, gy, gp = p.ct(x), p.ct(y), p.pt(pt)
            ptl = Plaintext(pt.m[:lvl], pt.scale)
            outs = [p.empty() for _ in range(4)]
            base = len(jobs)
            jobs += [dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=outs[0]),
                     dict(op=pf.PFT_JOB_SUB, a=gx, b=gy, out=outs[1]),
                     dict(op=pf.PFT_JOB_MUL_PLAIN, a=gx, p=gp, out=outs[2]),
                     dict(op=pf.PFT_JOB_MUL_PLAIN, a=outs[0], p=gp, out=outs[3], after=base)]
            s = o.add(x, y)
            checks += [(p, outs[0], s, "add"), (p, outs[1], o.sub(x, y), "sub"),
                       (p, outs[2], o.mul_plain(x, ptl), "mul_plain"), (p, outs[3], o.mul_plain(s, ptl), "after")]
    pf.pft_run_jobs(rings[0].ctx, jobs)
    pf.pft_device_status(rings[0].ctx)
    for p, h, want, what in checks:
        p.assert_equal(h, want, "%s N=%d level %d" % (what, p.N, want.c.shape[1]))


def test_serial_chain_across_rings(rings):
    """Each job adds y to the previous job's output: every tile waits for the whole previous job."""
    pf = rings[0].pft
    jobs, checks = [], []
    for p in rings:
        o = p.orc
        x, y, _ = operands(p, p.orc.L, 500 + p.N)
        gx, gy = p.ct(x), p.ct(y)
        want, prev = x, gx
        for k in range(12):
            out = p.empty()
            jobs.append(dict(op=pf.PFT_JOB_ADD, a=prev, b=gy, out=out, after=len(jobs) - 1 if k else -1))
            want = o.add(want, y)
            prev = out
        checks.append((p, prev, want))
    pf.pft_run_jobs(rings[0].ctx, jobs)
    pf.pft_device_status(rings[0].ctx)
    for p, h, want in checks:
        p.assert_equal(h, want, "chain of 12 at N=%d" % p.N)


def test_in_place_chain(rings):
    """out aliasing an input: x <- x + y, then x <- x - y (after) restores x."""
    p = rings[1]
    pf, o = p.pft, p.orc
    x, y, _ = operands(p, 4, 900)
    gx, gy = p.ct(x), p.ct(y)
    pf.pft_run_jobs(p.ctx, [dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=gx),
                           dict(op=pf.PFT_JOB_SUB, a=gx, b=gy, out=gx, after=0)])
    p.assert_equal(gx, o.sub(o.add(x, y), y), "in place")


def test_hazards_and_arguments(rings):
    a, b = rings
    pf = a.pft
    x, y, pt = operands(a, 3, 1000)
    gx, gy, gp = a.ct(x), a.ct(y), a.pt(pt)
    t, u = a.empty(), a.empty()
    bx = b.ct(operands(b, 3, 1100)[0])

    def code(jobs, timeout=1.0):
        with pytest.raises(pf.PftError) as e:
            pf.pft_run_jobs(a.ctx, jobs, timeout)
        return e.value.code

    # read after write without `after`
    assert code([dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=t), dict(op=pf.PFT_JOB_ADD, a=t, b=gy, out=u)]) == \
        pf.PFT_ERR_ARG
    # write after read without `after`
    assert code([dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=t), dict(op=pf.PFT_JOB_ADD, a=gy, b=gy, out=gx)]) == \
        pf.PFT_ERR_ARG
    # `after` must name an earlier job
    assert code([dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=t, after=0)]) == pf.PFT_ERR_ARG
    # operands of two rings, levels that differ, an unknown op, a timeout out of range
    assert code([dict(op=pf.PFT_JOB_ADD, a=gx, b=bx, out=t)]) == pf.PFT_ERR_ARG
    low = a.ct(a.orc.drop_level(y, 2))
    assert code([dict(op=pf.PFT_JOB_ADD, a=gx, b=low, out=t)]) == pf.PFT_ERR_LEVEL_MISMATCH
    assert code([dict(op=7, a=gx, b=gy, out=t)]) == pf.PFT_ERR_ARG
    assert code([dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=t)], timeout=0.0) == pf.PFT_ERR_ARG
    # a transitive dependency is enough: job 2 reads job 0's output through job 1
    pf.pft_run_jobs(a.ctx, [dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=t),
                            dict(op=pf.PFT_JOB_SUB, a=gx, b=gy, out=u, after=0),
                            dict(op=pf.PFT_JOB_ADD, a=t, b=u, out=u, after=1)])
    o = a.orc
    a.assert_equal(u, o.add(o.add(x, y), o.sub(x, y)), "transitive")
    # products take the scale of both factors; adding them to a sum is refused
    assert code([dict(op=pf.PFT_JOB_MUL_PLAIN, a=gx, p=gp, out=t),
                 dict(op=pf.PFT_JOB_ADD, a=t, b=gy, out=u, after=0)]) == pf.PFT_ERR_SCALE_MISMATCH
    pf.pft_run_jobs(a.ctx, [])  # empty list: nothing to do


def test_external_flag_released_and_expired(rings):
    import torch

    p = rings[0]
    pf, o = p.pft, p.orc
    x, y, _ = operands(p, 5, 1200)
    gx, gy = p.ct(x), p.ct(y)
    flag = torch.zeros(4, dtype=torch.int32, device="cuda")
    # released: the word already holds the value
    flag.fill_(3)
    out = p.empty()
    pf.pft_run_jobs(p.ctx, [dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=out, wait_flag=flag.data_ptr(), wait_value=3)])
    pf.pft_device_status(p.ctx)
    p.assert_equal(out, o.add(x, y), "released flag")
    # never released: every CTA gives up after 50 ms and the device flag reports it once
    flag.zero_()
    out2 = p.empty()
    pf.pft_run_jobs(p.ctx, [dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=out2, wait_flag=flag.data_ptr(), wait_value=1)],
                    0.05)
    with pytest.raises(pf.PftError) as e:
        pf.pft_device_status(p.ctx)
    assert e.value.code == pf.PFT_ERR_TIMEOUT
    pf.pft_device_status(p.ctx)  # cleared
    # the context keeps working
    out3 = p.empty()
    pf.pft_run_jobs(p.ctx, [dict(op=pf.PFT_JOB_SUB, a=gx, b=gy, out=out3)])
    p.assert_equal(out3, o.sub(x, y), "after the expired wait")
