"""Check of a neighbor list's reverse-pair index: for pair p = (i -> j, n), rev[p] must be the
pair (j -> i, -n) of j's list.  Each atom lists a (j, n) at most once, so these conditions fix
rev exactly; the check runs on the device (torch) to cover lists of 10^8 pairs."""
import torch


def check_reverse(api, nb, b):
    ex = api.mtp_nbr_export(nb, b, want_r=False)
    rev = api.mtp_nbr_reverse(nb).long()
    off, j, img = ex["off"], ex["j"].long(), ex["img"]
    n, P = off.numel() - 1, j.numel()
    assert rev.numel() == P
    if P == 0:
        return
    owner = torch.repeat_interleave(torch.arange(n, device=off.device), off[1:] - off[:-1])
    assert bool(((rev >= 0) & (rev < P)).all()), "reverse index out of range"
    assert torch.equal(j[rev], owner), "reverse pair has another center"
    assert torch.equal(img[rev], -img), "reverse pair has another image"
    assert torch.equal(rev[rev], torch.arange(P, device=rev.device)), "reverse is not an involution"
