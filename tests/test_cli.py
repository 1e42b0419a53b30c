"""The command-line front end's host-side behaviour (no GPU needed): usage,
and every malformed input rejected with exit status 2 and a message before
any device work."""
import subprocess

import pytest

from paper_2106_04034_gb300.build import CLI, build_library


@pytest.fixture(scope="module")
def cli():
    build_library()
    return CLI


def _run(cli, *args):
    return subprocess.run([cli, *args], capture_output=True, text=True, timeout=60)


def test_usage(cli):
    r = _run(cli, "-help")
    assert r.returncode == 0 and "train_file" in r.stderr
    r = _run(cli)
    assert r.returncode == 2 and "missing -train_file" in r.stderr
    r = _run(cli, "-bogus")
    assert r.returncode == 2 and "unknown" in r.stderr


@pytest.mark.parametrize("rows,msg", [
    ("1 2 3\n4 5\n", "columns"),                 # ragged
    ("1 2 nan\n", "finite"),                     # non-finite
    ("\n# only a comment\n", "no cases"),        # empty
    ("7\n", "feature"),                          # a target without features
])
def test_bad_case_files(cli, tmp_path, rows, msg):
    f = tmp_path / "train.txt"
    f.write_text(rows)
    r = _run(cli, "-train_file", str(f))
    assert r.returncode == 2 and msg in r.stderr, r.stderr


def test_test_file_must_match_features(cli, tmp_path):
    (tmp_path / "tr.txt").write_text("1 2 3\n4 5 6\n")
    (tmp_path / "te.txt").write_text("1 2\n")
    r = _run(cli, "-train_file", str(tmp_path / "tr.txt"), "-test_file", str(tmp_path / "te.txt"))
    assert r.returncode == 2 and "features" in r.stderr


@pytest.mark.parametrize("text,msg", [
    ("pop_size = 1\n", "pop_size"),              # rejected by gsgp_config_error
    ("colour = 3\n", "unknown key"),
    ("generations\n", "key = value"),
    ("ms = fast\n", "needs a number"),
    ("runs = 0\n", "runs"),
])
def test_bad_config(cli, tmp_path, text, msg):
    (tmp_path / "tr.txt").write_text("1 2 3\n4 5 6\n")
    (tmp_path / "c.ini").write_text("[gsgp]\n; comment\n" + text)
    r = _run(cli, "-train_file", str(tmp_path / "tr.txt"), "-config", str(tmp_path / "c.ini"))
    assert r.returncode == 2 and msg in r.stderr, r.stderr


def test_bad_model_file(cli, tmp_path):
    (tmp_path / "x.txt").write_text("1 2\n")
    (tmp_path / "m.txt").write_text("gsgp-model 7\n")
    r = _run(cli, "-model", str(tmp_path / "m.txt"), "-predict_file", str(tmp_path / "x.txt"))
    assert r.returncode == 2 and "version" in r.stderr
    r = _run(cli, "-model", str(tmp_path / "m.txt"))
    assert r.returncode == 2 and "predict_file" in r.stderr
