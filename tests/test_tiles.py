"""Phase-3 tile height of the persistent kernel (safr_set_tile_rows).

Every even height from 2 to min(32, M) is a valid tiling; most leave a ragged
last tile (M not a multiple of the height).  On mixed LGS + NGS plans each
tile stages the LGS source rows it needs, combines them into its output rows
on the spectra (the row half of the bilinear resample), then transforms one
row pair per complex FFT, so the heights exercise different source-row spans,
row pairings and odd final pairs.  The layers must match the FP64 oracle at
the precision's tolerance for every height, and returning to the cost
model's choice must give back the first result bit for bit.
"""
import pytest
from layer_errors import assert_layers

torch = pytest.importorskip("torch")


def test_set_tile_rows_rejects_bad_arguments_without_a_gpu():
    from paper_2510_19542_gb300 import safr
    lib = safr.load()
    for rows in (0, 2, 3, -2):
        assert lib.safr_set_tile_rows(None, rows) == safr.SAFR_ERR_INVALID_ARG


def _cases(synth):
    small = synth.scaled(synth.config(2), M=64, P=20)
    small64 = dict(synth.scaled(synth.config(2), M=32, P=10), precision="fp64")
    small64["name"] += "-fp64"
    big = synth.scaled(synth.config(2), M=512, P=160, L=6)  # 16 values per lane, B not staged
    return [small, small64, synth.config(2), big]


@pytest.mark.gpu
def test_every_tile_height_matches_the_oracle(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19542_gb300 import safr, synth
    for g in _cases(synth):
        fp64 = g.get("precision") == "fp64"
        tol = 1e-12 if fp64 else 1e-5
        x = synth.frame(g)
        ref = oracle_mod.OraclePlan(g).reconstruct(x)
        p = safr.Plan(g, device=0, path=safr.SAFR_PATH_FUSED)
        xin = torch.from_numpy(x).to("cuda:0", torch.float64 if fp64 else torch.float32)
        first = p.reconstruct(xin).clone()
        default_rows = safr.safr_get_plan_info(p.handle)["tile_rows"]
        M = g["M"]
        ran = []
        for rows in range(2, min(32, M) + 1, 2):
            try:
                safr.safr_set_tile_rows(p.handle, rows)
            except safr.SafrError as e:  # the tile does not fit in shared memory: choice unchanged
                assert e.status == safr.SAFR_ERR_UNSUPPORTED_SIZE, (g["name"], rows)
                continue
            assert safr.safr_get_plan_info(p.handle)["tile_rows"] == rows
            got = p.reconstruct(xin).double().cpu().numpy()
            assert safr.safr_get_status(p.handle) == 0, (g["name"], rows)
            assert_layers(got, ref, tol, (g["name"], rows))
            ran.append(rows)
        # heights with a ragged last tile and the cost model's own height were among them
        assert default_rows in ran and any(M % r for r in ran), (g["name"], ran)
        # values outside the range leave the choice as it was
        for bad in (1, 3, min(32, M) + 2, -2):
            with pytest.raises(safr.SafrError):
                safr.safr_set_tile_rows(p.handle, bad)
        assert safr.safr_get_plan_info(p.handle)["tile_rows"] == ran[-1]
        safr.safr_set_tile_rows(p.handle, 0)
        assert safr.safr_get_plan_info(p.handle)["tile_rows"] == default_rows
        assert torch.equal(p.reconstruct(xin), first), g["name"]
        p.close()
