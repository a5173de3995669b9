"""Helpers for the GPU tests: move generated events to the device and convert between the
oracle's track-major arrays and the library's structure-of-arrays planes."""
import math

import numpy as np

TRI = [(i, j) for i in range(6) for j in range(i + 1)]  # packed lower triangle, row order
# parity tolerances: |d| <= 1e-4 max(|ref|, floor) per parameter, chi2 |d| <= 1e-3 max(chi2, 1)
PAR_REL = 1e-4
PAR_FLOOR = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])
CHI2_REL = 1e-3


def device_hits(batch, device="cuda"):
    import torch
    from paper_1702_06359_gb300.tkf import DeviceHits
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(device)
    return DeviceHits(x=t(batch.x, torch.float32), y=t(batch.y, torch.float32), z=t(batch.z, torch.float32),
                      var_u=t(batch.var_u, torch.float32), var_v=t(batch.var_v, torch.float32),
                      layer=t(batch.layer, torch.int32), event_off=t(batch.hit_off, torch.int32))


def pack_cov(cov):
    """[n, 6, 6] -> [21, n]"""
    return np.stack([cov[:, i, j] for i, j in TRI], axis=0)


def unpack_cov(c21):
    """[21, n] -> [n, 6, 6]"""
    n = c21.shape[1]
    out = np.zeros((n, 6, 6))
    for k, (i, j) in enumerate(TRI):
        out[:, i, j] = c21[k]
        out[:, j, i] = c21[k]
    return out


def device_tracks(par, cov, chi2, nhits, hit_idx, event=None, precision=0, device="cuda"):
    """Oracle-layout arrays ([n, 6], [n, 6, 6], [n], [n], [n, L]) -> DeviceTracks planes."""
    import torch
    from paper_1702_06359_gb300.tkf import FP64, DeviceTracks
    dt = torch.float64 if precision == FP64 else torch.float32
    n = len(par)
    return DeviceTracks(
        par=torch.as_tensor(np.ascontiguousarray(par.T), dtype=dt).to(device),
        cov=torch.as_tensor(np.ascontiguousarray(pack_cov(cov)), dtype=dt).to(device),
        chi2=torch.as_tensor(np.asarray(chi2), dtype=dt).to(device),
        nhits=torch.as_tensor(np.asarray(nhits), dtype=torch.int32).to(device),
        hit_idx=torch.as_tensor(np.ascontiguousarray(np.asarray(hit_idx).T), dtype=torch.int32).to(device),
        event=torch.as_tensor(np.zeros(n) if event is None else np.asarray(event), dtype=torch.int32).to(device),
        n=n)


def host_tracks(t):
    """DeviceTracks -> dict of oracle-layout numpy arrays (FP64)."""
    n = t.n if t.n >= 0 else t.stride
    par = t.par.double().cpu().numpy()[:, :n].T.copy()
    cov = unpack_cov(t.cov.double().cpu().numpy()[:, :n])
    return dict(par=par, cov=cov, chi2=t.chi2.double().cpu().numpy()[:n], nhits=t.nhits.cpu().numpy()[:n],
                hit_idx=t.hit_idx.cpu().numpy()[:, :n].T.copy() if t.hit_idx is not None else None)


def rounded(a, precision):
    """The values the GPU sees: float32-rounded unless the mode is FP64."""
    from paper_1702_06359_gb300.tkf import FP64
    return np.asarray(a, dtype=np.float64) if precision == FP64 else np.asarray(a, dtype=np.float32).astype(np.float64)


def param_violations(got, ref, rel=PAR_REL):
    d = got - ref
    d[:, 4] = (d[:, 4] + math.pi) % (2 * math.pi) - math.pi
    bound = rel * np.maximum(np.abs(ref), PAR_FLOOR[None, :])
    return np.abs(d) > bound, np.max(np.abs(d) / bound) if len(d) else 0.0


def chi2_violations(got, ref, rel=CHI2_REL):
    bound = rel * np.maximum(np.abs(ref), 1.0)
    return np.abs(got - ref) > bound, np.max(np.abs(got - ref) / bound) if len(ref) else 0.0


def divergence_allowed(got_hits, ref, s, tol=1e-3):
    """Whether a GPU hit list that differs from the oracle's best for seed s is explained by a
    fragile decision (the parity definition's exemption: two chi2 values within `tol` of each other or
    of the cut).  `ref` is the oracle's BuildResult.  Either the lists first differ at or after
    the oracle's first fragile layer, or the GPU's track is one of the oracle's final candidates
    with as many hits as the best and a total chi2 within `tol` of it (a near-tie in the final
    ranking between candidates that branched earlier)."""
    d = int(np.argmax(got_hits != ref.hits[s, 0]))
    if d >= ref.fragile[s]:
        return True
    for k in range(1, min(int(ref.n_cand[s]), ref.hits.shape[1])):
        if (np.array_equal(got_hits, ref.hits[s, k]) and ref.nhits[s, k] == ref.nhits[s, 0]
                and abs(ref.chi2[s, k] - ref.chi2[s, 0]) <= tol * max(abs(ref.chi2[s, 0]), 1.0)):
            return True
    return False
