"""The configuration runner's validation (host logic, no GPU)."""
import pytest

from paper_2109_02598_gb300.run import ConfigError, validate


def base():
    return {"grid": {"shape": [64, 64]},
            "model": {"name": "ch", "coeffs": [1, 1, 1], "dt": 0.01},
            "init": {"synthetic": "cahn_hilliard_init", "args": {"seed": 2}},
            "run": {"steps": 100}}


def test_defaults_filled():
    c = validate(base())
    assert c["grid"]["h"] == 1.0 and c["model"]["stencil"] == "std"
    assert c["run"]["tuning"] == "auto" and c["run"]["series_every"] == 100
    assert c["run"]["checkpoint_every"] == 0 and c["run"]["energy"] is False


@pytest.mark.parametrize("edit,msg", [
    (lambda c: c.pop("run"), "missing section"),
    (lambda c: c["grid"].update(shape=[64]), "grid.shape"),
    (lambda c: c["grid"].update(shape=[64, -1]), "grid.shape"),
    (lambda c: c["model"].update(name="xy"), "model.name"),
    (lambda c: c["model"].pop("dt"), "dt"),
    (lambda c: c["init"].update(npy=["a.npy"]), "exactly one"),
    (lambda c: c.update(init={"npy": ["a.npy"]}), "2 files|1 files|must list"),
    (lambda c: c["run"].update(steps=-1), "run.steps"),
    (lambda c: c["run"].update(tuning=[1, 2]), "run.tuning"),
    (lambda c: c["run"].update(series_every=0), "series_every"),
])
def test_rejections(edit, msg):
    c = base()
    edit(c)
    if msg == "2 files|1 files|must list":
        c["model"]["name"] = "gs"  # two fields, one file given
        c["model"]["coeffs"] = [0.2, 0.1, 0.04, 0.06]
        msg = "must list"
    with pytest.raises(ConfigError, match=msg):
        validate(c)


def test_command_line_reports_configuration_errors(tmp_path, capsys):
    import json

    from paper_2109_02598_gb300.run import main
    assert main([]) == 2  # usage
    bad = base()
    bad["model"]["name"] = "nope"
    p = tmp_path / "bad.json"
    p.write_text(json.dumps(bad))
    assert main([str(p)]) == 2
    assert "configuration error" in capsys.readouterr().err
