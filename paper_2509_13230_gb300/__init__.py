"""GB300-native Miller-Hagberg sampling of maximum-entropy network models
(Li, Wang, Kojaku, arXiv 2509.13230)."""
