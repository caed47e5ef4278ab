"""Index arithmetic of the TMA sweep's copy ring (k_fused.cu, sweep_body),
restated on the host: which copies can still be in flight when a block
gives up on a wait, and which stage and mbarrier parity each of them
completes.  The kernel's abort path drains the last NST issues, issue t at
stage t % NST with parity (t / NST) & 1; this checks that this set covers
every copy that can still land, for every ring depth, step count and step
at which the first wait can fail."""
import pytest


def ring_run(total, nst, abort_at):
    """Issue/consume order of the kernel: NST issues up front, then after the
    barrier of every consumed step one refill into the stage just released,
    unless a wait has failed.  Returns the issues (t, stage, parity), the
    copies that may be in flight at the end and the issue count."""
    issues = []
    stage_uses = [0] * nst

    def issue(t, stage):
        assert stage == t % nst
        issues.append((t, stage, stage_uses[stage] & 1))
        stage_uses[stage] += 1

    n = 0
    for t in range(min(nst, total)):
        issue(t, t)
        n += 1
    q, ph = 0, 0
    pending = set(range(n))
    for step in range(total):
        if step < abort_at:
            # the wait of this step succeeds: it waited on its own issue
            t, stage, par = issues[step]
            assert (stage, par) == (q, ph)
            pending.discard(step)
            if n < total:
                issue(n, q)
                pending.add(n)
                n += 1
        q += 1
        if q == nst:
            q, ph = 0, ph ^ 1
    return issues, pending, n


@pytest.mark.parametrize("nst", [2, 3, 4])
@pytest.mark.parametrize("total", [1, 2, 5, 13, 66, 390])
def test_abort_drain_covers_every_copy_in_flight(nst, total):
    for abort_at in list(range(min(total, 8))) + [total // 2, total - 1]:
        issues, pending, n = ring_run(total, nst, abort_at)
        drain = list(range(max(0, n - nst), n))
        assert pending <= set(drain), (abort_at, pending, drain)
        stages = [t % nst for t in drain]
        assert len(set(stages)) == len(stages)          # one pending phase per stage
        for t in drain:
            _, stage, par = issues[t]
            assert (stage, par) == (t % nst, (t // nst) & 1)
